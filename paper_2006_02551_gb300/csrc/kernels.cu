// DGTD stage kernels for sm_103a: one fused launch per element class and
// Runge-Kutta stage computes the right-hand side of the semi-discrete
// system and applies the low-storage Runge-Kutta update.
//
// Per element (Section II.A):
//   * face traces through the neighbour map and the upwind flux,
//   * volume curl through the reference differentiation matrices and the
//     metric terms, LIFT of the scaled flux (curl operator Cbar_k),
//   * in PML elements the weight-adjusted terms of eqs. 26-29: interpolate
//     E, H, P^E, P^H to the quadrature nodes (V_q), form the CPML tensors of
//     eq. 9 pointwise from the stored sigma_u (kappa_u) samples, project
//     back (P_q); with kappa = 1 the outer P_q a^{-1} V_q is the identity
//     (a = 1 and P_q V_q = I), otherwise it is applied explicitly,
//   * res <- A res + dt rhs, q <- q + B res.
// The tile of T elements lives in shared memory; threads sweep it in
// (element, node) or (element, quadrature node) order.
#include "kernels.cuh"

#include <cstdio>

namespace wadg {

template <int N>
struct Dims {
  static constexpr int Np = (N + 1) * (N + 2) * (N + 3) / 6;
  static constexpr int Nfp = (N + 1) * (N + 2) / 2;
  static constexpr int Nq = (N + 1) * (N + 1) * (N + 1);
  static constexpr int NF = 4 * Nfp;
};

constexpr int kThreads = 256;

template <typename Real, int N, bool PML>
struct Tile {
  using D = Dims<N>;
  static constexpr int per_elem_std = 6 * D::Np + 6 * D::NF + 16 + 9;
  static constexpr int big_pml = (6 * D::NF > 12 * D::Nq) ? 6 * D::NF : 12 * D::Nq;
  static constexpr int per_elem_pml = 18 * D::Np + big_pml + 16 + 9;
  static constexpr int per_elem = PML ? per_elem_pml : per_elem_std;
  static constexpr int budget = 96 * 1024;
  static constexpr int t0 = budget / (per_elem * (int)sizeof(Real));
  static constexpr int T = t0 < 1 ? 1 : (t0 > 32 ? 32 : t0);
  static constexpr size_t smem = (size_t)T * per_elem * sizeof(Real) + 64 * sizeof(int);
};

__device__ __forceinline__ double dipole_current(const SrcDev& s, double t) {
  double tau = s.width;
  double g = exp(-(t - s.t0) * (t - s.t0) / (4.0 * tau * tau));
  return s.amp * (-(t - s.t0) / (2.0 * tau * tau)) * g;
}

template <typename Real, int N, bool PML, bool KAPPA>
__global__ void __launch_bounds__(kThreads)
stage_kernel(const StageParams<Real> P) {
  using D = Dims<N>;
  constexpr int Np = D::Np, Nfp = D::Nfp, Nq = D::Nq, NF = D::NF;
  using TL = Tile<Real, N, PML>;
  constexpr int T = TL::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  Real* qs = sm;                          // [T][6][Np]
  Real* ps = qs + T * 6 * Np;             // [T][6][Np]   (PML)
  Real* rs = ps + (PML ? T * 6 * Np : 0); // [T][6][Np]   (PML)
  Real* big = rs + (PML ? T * 6 * Np : 0);// flux [T][6][NF] / tz [T][12][Nq]
  Real* fl = big;
  Real* nrm = big + T * (PML ? TL::big_pml : 6 * NF);  // [T][4][4]
  Real* met = nrm + T * 16;                             // [T][9]
  int* srcl = reinterpret_cast<int*>(met + T * 9);      // [64]
  __shared__ int nsl;

  const Real* DrT = P.ops;
  const Real* DsT = DrT + Np * Np;
  const Real* DtT = DsT + Np * Np;
  const Real* LIFTT = DtT + Np * Np;
  const Real* VqT = LIFTT + NF * Np;
  const Real* PqT = VqT + Np * Nq;
  const unsigned char* Fmask = P.tabs;
  const unsigned char* fperm = P.tabs + NF;

  const int tid = threadIdx.x;
  const int b = blockIdx.y;
  const int t0 = blockIdx.x * T;
  if (t0 >= P.n_elem) return;
  const int ne = min(T, P.n_elem - t0);
  const int eg0 = P.e_begin + t0;           // internal id of the first element
  const Real* qin = P.qin + (int64_t)b * P.strideQ;
  Real* qout = P.qout + (int64_t)b * P.strideQ;
  Real* resq = P.resq + (int64_t)b * P.strideQ;
  const double tbase = P.t_dev ? *P.t_dev : P.t;
  const double tst = tbase + P.rk_c * P.dt;
  const Real rka = (Real)P.rk_a, rkb = (Real)P.rk_b, rdt = (Real)P.dt;

  // ---- phase 0: fields, geometry, sources of this tile
  if (tid == 0) nsl = 0;
  for (int idx = tid; idx < ne * 6 * Np; idx += kThreads)
    qs[idx] = qin[(int64_t)eg0 * 6 * Np + idx];
  if (PML) {
    const Real* pin = P.p + (int64_t)b * P.strideP + (int64_t)(eg0 - P.K0) * 6 * Np;
    for (int idx = tid; idx < ne * 6 * Np; idx += kThreads) ps[idx] = pin[idx];
  }
  for (int idx = tid; idx < ne * 4; idx += kThreads) {
    int e = idx >> 2, f = idx & 3;
    const double* g = P.geo + (int64_t)(eg0 + e) * 9;
    double gx, gy, gz;
    if (f == 0) { gx = -g[6]; gy = -g[7]; gz = -g[8]; }
    else if (f == 1) { gx = -g[3]; gy = -g[4]; gz = -g[5]; }
    else if (f == 2) { gx = g[0] + g[3] + g[6]; gy = g[1] + g[4] + g[7]; gz = g[2] + g[5] + g[8]; }
    else { gx = -g[0]; gy = -g[1]; gz = -g[2]; }
    double mag = sqrt(gx * gx + gy * gy + gz * gz);
    Real* nn = nrm + (e * 4 + f) * 4;
    nn[0] = (Real)(gx / mag); nn[1] = (Real)(gy / mag); nn[2] = (Real)(gz / mag);
    nn[3] = (Real)mag;   // Fscale = sJ / J = |grad of the face coordinate|
  }
  for (int idx = tid; idx < ne * 9; idx += kThreads)
    met[idx] = (Real)P.geo[(int64_t)eg0 * 9 + idx];
  __syncthreads();
  for (int s = tid; s < P.nsrc; s += kThreads) {
    const SrcDev& sd = P.src[s];
    if (sd.batch == b && sd.elem >= eg0 && sd.elem < eg0 + ne) {
      int slot = atomicAdd(&nsl, 1);
      if (slot < 64) srcl[slot] = s;
    }
  }

  // ---- phase 1: upwind flux at the 4 Nfp trace nodes (scaled by Fscale)
  for (int idx = tid; idx < ne * NF; idx += kThreads) {
    const int e = idx / NF, fm = idx - e * NF;
    const int f = fm / Nfp, m = fm - f * Nfp;
    const int eg = eg0 + e;
    const int ni = Fmask[fm];
    const Real* nn = nrm + (e * 4 + f) * 4;
    const Real nx = nn[0], ny = nn[1], nz = nn[2], fsc = nn[3];
    Real Em[3], Hm[3], Ep[3], Hp[3];
    for (int c = 0; c < 3; ++c) {
      Em[c] = qs[(e * 6 + c) * Np + ni];
      Hm[c] = qs[(e * 6 + 3 + c) * Np + ni];
    }
    const Real ZM = P.mat[eg * 3 + 2];
    Real ZP = ZM;
    const int nb = P.nbr[eg * 4 + f];
    if (nb >= 0) {
      const int code = P.code[eg * 4 + f];
      const int np2 = fperm[(f * 24 + code) * Nfp + m];
      const Real* qn = qin + (int64_t)nb * 6 * Np + np2;
      for (int c = 0; c < 3; ++c) {
        Ep[c] = qn[c * Np];
        Hp[c] = qn[(3 + c) * Np];
      }
      ZP = P.mat[nb * 3 + 2];
    } else {   // perfect electric conductor: mirror state
      for (int c = 0; c < 3; ++c) { Ep[c] = -Em[c]; Hp[c] = Hm[c]; }
    }
    const Real dEx = Ep[0] - Em[0], dEy = Ep[1] - Em[1], dEz = Ep[2] - Em[2];
    const Real dHx = Hp[0] - Hm[0], dHy = Hp[1] - Hm[1], dHz = Hp[2] - Hm[2];
    const Real ndE = nx * dEx + ny * dEy + nz * dEz;
    const Real ndH = nx * dHx + ny * dHy + nz * dHz;
    // n x dH, n x (n x dE) = n (n.dE) - dE
    const Real cHx = ny * dHz - nz * dHy, cHy = nz * dHx - nx * dHz, cHz = nx * dHy - ny * dHx;
    const Real cEx = ny * dEz - nz * dEy, cEy = nz * dEx - nx * dEz, cEz = nx * dEy - ny * dEx;
    const Real al = (Real)P.alpha;
    const Real YM = Real(1) / ZM, YP = Real(1) / ZP;
    const Real sH = fsc / (ZM + ZP), sE = fsc / (YM + YP);
    Real* fe = fl + e * 6 * NF + fm;
    // drives E: (Z+ n x dH - alpha n x (n x dE)) / (Z- + Z+)
    fe[0 * NF] = sH * (ZP * cHx - al * (nx * ndE - dEx));
    fe[1 * NF] = sH * (ZP * cHy - al * (ny * ndE - dEy));
    fe[2 * NF] = sH * (ZP * cHz - al * (nz * ndE - dEz));
    // drives H: (Y+ n x dE + alpha n x (n x dH)) / (Y- + Y+)
    fe[3 * NF] = sE * (YP * cEx + al * (nx * ndH - dHx));
    fe[4 * NF] = sE * (YP * cEy + al * (ny * ndH - dHy));
    fe[5 * NF] = sE * (YP * cEz + al * (nz * ndH - dHz));
  }
  __syncthreads();
  const int nsrc_l = min(nsl, 64);

  // ---- phase 2: volume curl + LIFT  ->  Cbar(H) (E rows), Cbar(E) (H rows)
  for (int idx = tid; idx < ne * Np; idx += kThreads) {
    const int e = idx / Np, i = idx - e * Np;
    const int eg = eg0 + e;
    Real dr[6], ds[6], dt[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) { dr[c] = 0; ds[c] = 0; dt[c] = 0; }
    const Real* qe = qs + e * 6 * Np;
    for (int j = 0; j < Np; ++j) {
      const Real a = DrT[j * Np + i], bb = DsT[j * Np + i], cc = DtT[j * Np + i];
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        const Real v = qe[c * Np + j];
        dr[c] += a * v; ds[c] += bb * v; dt[c] += cc * v;
      }
    }
    const Real* g = met + e * 9;
    Real dx[6], dy[6], dz[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      dx[c] = g[0] * dr[c] + g[3] * ds[c] + g[6] * dt[c];
      dy[c] = g[1] * dr[c] + g[4] * ds[c] + g[7] * dt[c];
      dz[c] = g[2] * dr[c] + g[5] * ds[c] + g[8] * dt[c];
    }
    Real lf[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) lf[c] = 0;
    const Real* fe = fl + e * 6 * NF;
    for (int fm = 0; fm < NF; ++fm) {
      const Real L = LIFTT[fm * Np + i];
#pragma unroll
      for (int c = 0; c < 6; ++c) lf[c] += L * fe[c * NF + fm];
    }
    // Cbar(H) = curl H + LIFT flux  (E rows); Cbar(E) = curl E + LIFT flux (H rows)
    Real CH[3], CE[3];
    CH[0] = dy[5] - dz[4] + lf[0];
    CH[1] = dz[3] - dx[5] + lf[1];
    CH[2] = dx[4] - dy[3] + lf[2];
    CE[0] = dy[2] - dz[1] + lf[3];
    CE[1] = dz[0] - dx[2] + lf[4];
    CE[2] = dx[1] - dy[0] + lf[5];
    for (int s = 0; s < nsrc_l; ++s) {
      const SrcDev& sd = P.src[srcl[s]];
      if (sd.elem != eg) continue;
      const Real jt = (Real)dipole_current(sd, tst);
      const Real w = P.src_w[srcl[s] * Np + i];
      CH[0] -= jt * (Real)sd.dir[0] * w;
      CH[1] -= jt * (Real)sd.dir[1] * w;
      CH[2] -= jt * (Real)sd.dir[2] * w;
    }
    const Real ie = P.mat[eg * 3 + 0], im = P.mat[eg * 3 + 1];
    Real rhs[6];
    rhs[0] = ie * CH[0]; rhs[1] = ie * CH[1]; rhs[2] = ie * CH[2];
    rhs[3] = -im * CE[0]; rhs[4] = -im * CE[1]; rhs[5] = -im * CE[2];
    if (!PML) {
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        const int64_t gi = ((int64_t)eg * 6 + c) * Np + i;
        Real r = rka * resq[gi] + rdt * rhs[c];
        resq[gi] = r;
        qout[gi] = qe[c * Np + i] + rkb * r;
      }
    } else {
#pragma unroll
      for (int c = 0; c < 6; ++c) rs[(e * 6 + c) * Np + i] = rhs[c];
    }
  }
  if (!PML) return;
  __syncthreads();

  // ---- phase 3: quadrature-node values and the pointwise CPML terms
  const int ep0 = eg0 - P.K0;
  Real* tz = big;  // [T][12][Nq]
  const Real ie0 = Real(1) / (Real)P.eps0;
  for (int idx = tid; idx < ne * Nq; idx += kThreads) {
    const int e = idx / Nq, qp = idx - e * Nq;
    Real v[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) v[c] = 0;
    const Real* qe = qs + e * 6 * Np;
    const Real* pe = ps + e * 6 * Np;
    for (int j = 0; j < Np; ++j) {
      const Real w = VqT[j * Nq + qp];
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        v[c] += w * qe[c * Np + j];
        v[6 + c] += w * pe[c * Np + j];
      }
    }
    const Real* sg = P.sig + (int64_t)(ep0 + e) * 3 * Nq + qp;
    Real sig[3] = {sg[0], sg[Nq], sg[2 * Nq]};
    Real kap[3] = {Real(1), Real(1), Real(1)};
    if (KAPPA) {
      const Real* kp = P.kap + (int64_t)(ep0 + e) * 3 * Nq + qp;
      kap[0] = kp[0]; kap[1] = kp[Nq]; kap[2] = kp[2 * Nq];
    }
    Real* tze = tz + e * 12 * Nq + qp;
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      const int vv = (u + 1) % 3, ww = (u + 2) % 3;
      // eq. 9
      const Real a = kap[vv] * kap[ww] / kap[u];
      const Real bc = (sig[vv] * kap[ww] + sig[ww] * kap[vv] - a * sig[u]) / kap[u] * ie0;
      const Real cc = sig[vv] * sig[ww] * ie0 * ie0 - bc * sig[u] * ie0;
      const Real dd = sig[u] / kap[u] * ie0;
      const Real ki = Real(1) / kap[u];
      tze[u * Nq] = bc * v[u] + cc * v[6 + u];                   // E:  b V E + c V P^E
      tze[(3 + u) * Nq] = bc * v[3 + u] + cc * v[9 + u];         // H:  b V H + c V P^H
      tze[(6 + u) * Nq] = ki * v[u] - dd * v[6 + u];             // P^E: k^-1 V E - d V P^E
      tze[(9 + u) * Nq] = ki * v[3 + u] - dd * v[9 + u];         // P^H
    }
  }
  __syncthreads();

  // ---- phase 4: projections P_q; finish eqs. 26-29 (kappa = 1) or P^E, P^H
  Real* pout = P.p + (int64_t)b * P.strideP;
  Real* resp = P.resp + (int64_t)b * P.strideP;
  for (int idx = tid; idx < ne * Np; idx += kThreads) {
    const int e = idx / Np, i = idx - e * Np;
    const int eg = eg0 + e;
    Real s[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) s[c] = 0;
    const Real* tze = tz + e * 12 * Nq;
    for (int qp = 0; qp < Nq; ++qp) {
      const Real w = PqT[qp * Np + i];
#pragma unroll
      for (int c = 0; c < 12; ++c) s[c] += w * tze[c * Nq + qp];
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const Real wv = rs[(e * 6 + c) * Np + i] - s[c];
      if (!KAPPA) {
        const int64_t gi = ((int64_t)eg * 6 + c) * Np + i;
        Real r = rka * resq[gi] + rdt * wv;
        resq[gi] = r;
        qout[gi] = qs[(e * 6 + c) * Np + i] + rkb * r;
      } else {
        rs[(e * 6 + c) * Np + i] = wv;
      }
      const int64_t pi = ((int64_t)(eg - P.K0) * 6 + c) * Np + i;
      Real r = rka * resp[pi] + rdt * s[6 + c];
      resp[pi] = r;
      pout[pi] = ps[(e * 6 + c) * Np + i] + rkb * r;
    }
  }
  if (!KAPPA) return;
  __syncthreads();

  // ---- phase 5: a^{-1} V_q applied to (Cbar/eps - s), kappa != 1
  for (int idx = tid; idx < ne * Nq; idx += kThreads) {
    const int e = idx / Nq, qp = idx - e * Nq;
    Real v[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) v[c] = 0;
    const Real* re = rs + e * 6 * Np;
    for (int j = 0; j < Np; ++j) {
      const Real w = VqT[j * Nq + qp];
#pragma unroll
      for (int c = 0; c < 6; ++c) v[c] += w * re[c * Np + j];
    }
    const Real* kp = P.kap + (int64_t)(ep0 + e) * 3 * Nq + qp;
    Real kap[3] = {kp[0], kp[Nq], kp[2 * Nq]};
    Real* tze = tz + e * 12 * Nq + qp;
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      const Real ainv = kap[u] / (kap[(u + 1) % 3] * kap[(u + 2) % 3]);
      tze[u * Nq] = ainv * v[u];
      tze[(3 + u) * Nq] = ainv * v[3 + u];
    }
  }
  __syncthreads();

  // ---- phase 6: P_q back to the nodes, E/H update
  for (int idx = tid; idx < ne * Np; idx += kThreads) {
    const int e = idx / Np, i = idx - e * Np;
    const int eg = eg0 + e;
    Real s[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) s[c] = 0;
    const Real* tze = tz + e * 12 * Nq;
    for (int qp = 0; qp < Nq; ++qp) {
      const Real w = PqT[qp * Np + i];
#pragma unroll
      for (int c = 0; c < 6; ++c) s[c] += w * tze[c * Nq + qp];
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const int64_t gi = ((int64_t)eg * 6 + c) * Np + i;
      Real r = rka * resq[gi] + rdt * s[c];
      resq[gi] = r;
      qout[gi] = qs[(e * 6 + c) * Np + i] + rkb * r;
    }
  }
}

template <typename Real, int N, bool PML, bool KAPPA>
static cudaError_t configure_one() {
  using TL = Tile<Real, N, PML>;
  return cudaFuncSetAttribute(stage_kernel<Real, N, PML, KAPPA>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TL::smem);
}

template <typename Real, int N, bool PML, bool KAPPA>
static cudaError_t launch_one(const StageParams<Real>& P, int nb, cudaStream_t s) {
  using TL = Tile<Real, N, PML>;
  if (P.n_elem <= 0) return cudaSuccess;
  dim3 grid((P.n_elem + TL::T - 1) / TL::T, nb);
  stage_kernel<Real, N, PML, KAPPA><<<grid, kThreads, TL::smem, s>>>(P);
  return cudaGetLastError();
}

template <typename Real, int N>
static cudaError_t configure_n() {
  cudaError_t e = configure_one<Real, N, false, false>();
  if (e == cudaSuccess) e = configure_one<Real, N, true, false>();
  if (e == cudaSuccess) e = configure_one<Real, N, true, true>();
  return e;
}

template <typename Real>
cudaError_t configure_stage_kernels(int N) {
  switch (N) {
    case 1: return configure_n<Real, 1>();
    case 2: return configure_n<Real, 2>();
    case 3: return configure_n<Real, 3>();
    case 4: return configure_n<Real, 4>();
    case 5: return configure_n<Real, 5>();
    default: return cudaErrorInvalidValue;
  }
}
template cudaError_t configure_stage_kernels<double>(int);
template cudaError_t configure_stage_kernels<float>(int);

template <typename Real, int N>
static cudaError_t dispatch_pml(bool pml, bool kappa, const StageParams<Real>& P, int nb,
                                cudaStream_t s) {
  if (!pml) return launch_one<Real, N, false, false>(P, nb, s);
  if (kappa) return launch_one<Real, N, true, true>(P, nb, s);
  return launch_one<Real, N, true, false>(P, nb, s);
}

template <typename Real>
cudaError_t launch_stage(int N, bool pml, bool kappa, const StageParams<Real>& P, int nb,
                         cudaStream_t s) {
  switch (N) {
    case 1: return dispatch_pml<Real, 1>(pml, kappa, P, nb, s);
    case 2: return dispatch_pml<Real, 2>(pml, kappa, P, nb, s);
    case 3: return dispatch_pml<Real, 3>(pml, kappa, P, nb, s);
    case 4: return dispatch_pml<Real, 4>(pml, kappa, P, nb, s);
    case 5: return dispatch_pml<Real, 5>(pml, kappa, P, nb, s);
    default: return cudaErrorInvalidValue;
  }
}
template cudaError_t launch_stage<double>(int, bool, bool, const StageParams<double>&, int,
                                          cudaStream_t);
template cudaError_t launch_stage<float>(int, bool, bool, const StageParams<float>&, int,
                                         cudaStream_t);

// ------------------------------------------------------------------ probes
template <typename Real>
__global__ void probe_kernel(const ProbeParams P) {
  const int p = blockIdx.x, b = blockIdx.y, lane = threadIdx.x;
  const Real* q = reinterpret_cast<const Real*>(P.q) + (int64_t)b * P.strideQ +
                  (int64_t)P.elem[p] * 6 * P.Np;
  const double* ell = P.ell + (int64_t)p * P.Np;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int i = lane; i < P.Np; i += 32) {
    const double l = ell[i];
#pragma unroll
    for (int c = 0; c < 6; ++c) acc[c] += l * (double)q[c * P.Np + i];
  }
#pragma unroll
  for (int c = 0; c < 6; ++c)
    for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
  if (lane == 0) {
    const int64_t st = *P.step;
    double* o = P.out + ((st * P.nprobe + p) * 6) * P.nb + b;
    for (int c = 0; c < 6; ++c) o[c * P.nb] = acc[c];
    atomicAdd(&P.obj[b], acc[0] * acc[0] + acc[1] * acc[1] + acc[2] * acc[2]);
  }
}

cudaError_t launch_probes(bool fp64, const ProbeParams& P, cudaStream_t s) {
  if (P.nprobe <= 0) return cudaSuccess;
  dim3 grid(P.nprobe, P.nb);
  if (fp64) probe_kernel<double><<<grid, 32, 0, s>>>(P);
  else probe_kernel<float><<<grid, 32, 0, s>>>(P);
  return cudaGetLastError();
}

__global__ void advance_kernel(double* t, int64_t* step, double dt) {
  *t += dt;
  *step += 1;
}

cudaError_t launch_advance(double* t_dev, int64_t* step_dev, double dt, cudaStream_t s) {
  advance_kernel<<<1, 1, 0, s>>>(t_dev, step_dev, dt);
  return cudaGetLastError();
}

// ---------------------------------------------------------- set-up kernels
// sigma_u, kappa_u at the quadrature nodes of every PML element, in double.
// prof: u0[3], L[3], sigma_max[3], p_sigma[3], kappa_max[3], eps0
template <typename Real>
__global__ void pml_samples_kernel(int Nq, int K1, int K0, const double* verts,
                                   const double* rq, const double* prof, Real* sig,
                                   Real* kap) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)K1 * Nq) return;
  const int e = (int)(idx / Nq), q = (int)(idx - (int64_t)e * Nq);
  const double* v = verts + (int64_t)(K0 + e) * 12;
  const double r = rq[q * 3], s = rq[q * 3 + 1], t = rq[q * 3 + 2];
  const double l0 = -0.5 * (1 + r + s + t), l1 = 0.5 * (1 + r), l2 = 0.5 * (1 + s),
               l3 = 0.5 * (1 + t);
  for (int u = 0; u < 3; ++u) {
    const double x = l0 * v[u] + l1 * v[3 + u] + l2 * v[6 + u] + l3 * v[9 + u];
    const double d = (fabs(x) - prof[u]) / prof[3 + u];
    double g = 0.0;
    if (d > 0) g = pow(d, prof[9 + u]);
    sig[((int64_t)e * 3 + u) * Nq + q] = (Real)(prof[6 + u] * g);
    if (kap) kap[((int64_t)e * 3 + u) * Nq + q] = (Real)(1.0 + (prof[12 + u] - 1.0) * g);
  }
}

template <typename Real>
cudaError_t launch_pml_samples(int Nq, int K1, int K0, const double* verts, const double* rq,
                               const double* prof, Real* sig, Real* kap, cudaStream_t s) {
  const int64_t n = (int64_t)K1 * Nq;
  if (n == 0) return cudaSuccess;
  const int th = 256;
  pml_samples_kernel<Real><<<(unsigned)((n + th - 1) / th), th, 0, s>>>(Nq, K1, K0, verts, rq,
                                                                       prof, sig, kap);
  return cudaGetLastError();
}
template cudaError_t launch_pml_samples<double>(int, int, int, const double*, const double*,
                                                const double*, double*, double*, cudaStream_t);
template cudaError_t launch_pml_samples<float>(int, int, int, const double*, const double*,
                                               const double*, float*, float*, cudaStream_t);

template <typename Real>
__global__ void check_finite_kernel(const Real* a, int64_t n, int* flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (!isfinite((double)a[i])) {
      *flag = 1;
      return;
    }
  }
}

template <typename Real>
cudaError_t launch_check_finite(const Real* a, int64_t n, int* flag, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  check_finite_kernel<Real><<<152 * 4, 256, 0, s>>>(a, n, flag);
  return cudaGetLastError();
}
template cudaError_t launch_check_finite<double>(const double*, int64_t, int*, cudaStream_t);
template cudaError_t launch_check_finite<float>(const float*, int64_t, int*, cudaStream_t);

}  // namespace wadg
