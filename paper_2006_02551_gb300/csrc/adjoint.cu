// Discrete adjoint of the Runge-Kutta stage (CUDA cores, FP64 or FP32),
// for the gradient of the probe objective J = sum_steps sum_probes |E(x_p)|^2
// with respect to the per-element permittivity eps_k and the PML profile
// parameters (sigma_max, p_sigma per axis), kappa = 1.
//
// Forward stage i: res_i = A_i res_{i-1} + dt f(q_in, t_i), q_out = q_in + B_i res_i,
// f = L q + source (curl with upwind flux, eqs. 26-29).  Reverse stage i,
// with lambda the adjoint of q and rho the adjoint of res:
//     mu = rho + B_i lambda_out
//     lambda_in = lambda_out + dt L^T mu,   rho_prev = A_i mu,
//     dJ/dtheta += dt mu . (df/dtheta)(q_in, t_i).
// L^T needs the neighbours' share of the face terms, so a reverse stage is two
// launches: adj_lift computes g = Fscale * LIFT^T (mu_E/eps, -mu_H/mu) at the
// trace nodes of every element (a scratch array), adj_main gathers the own and
// the neighbour's g to transpose the upwind flux, applies curl^T, V_q^T, P_q^T,
// and accumulates the parameter derivatives.
#include "kernels.cuh"

#include <cstdio>

namespace wadg {

namespace {

template <int N, int QC = 0>
struct AD {
  static constexpr int Np = (N + 1) * (N + 2) * (N + 3) / 6;
  static constexpr int Nfp = (N + 1) * (N + 2) / 2;
  static constexpr int NF = 4 * Nfp;
  static constexpr int Nq = quad_capacity(N, QC);   // volume quadrature points
  static constexpr int NpP = (Np + 3) & ~3;
  static constexpr int NqP = (Nq + 3) & ~3;
};

constexpr int kAdjThreads = 256;

template <typename Real>
__device__ __forceinline__ void cross3(const Real* n, const Real* a, Real* o) {
  o[0] = n[1] * a[2] - n[2] * a[1];
  o[1] = n[2] * a[0] - n[0] * a[2];
  o[2] = n[0] * a[1] - n[1] * a[0];
}

// ---------------------------------------------------------------- adj_lift
// G[b][e][fm][0..2] = Fscale * (LIFT^T (mu_E / eps))[fm]   (transpose of the E-row flux)
// G[b][e][fm][3..5] = Fscale * (LIFT^T (-mu_H / mu))[fm]   (transpose of the H-row flux)
template <typename Real, int N>
__global__ void __launch_bounds__(kAdjThreads) adj_lift_kernel(const AdjParams<Real> A) {
  using D = AD<N>;
  constexpr int Np = D::Np, NF = D::NF, NpP = D::NpP, Nfp = D::Nfp;
  constexpr int T = 8;
  __shared__ Real a[T][6][Np];
  const int tid = threadIdx.x, b = blockIdx.y;
  const int e0 = blockIdx.x * T;
  if (e0 >= A.K) return;
  const int ne = min(T, A.K - e0);
  const Real* lam = A.lam_q + (int64_t)b * A.strideQ;
  const Real* rho = A.rho_q + (int64_t)b * A.strideQ;
  const Real Bi = A.rk_b_r;
  for (int idx = tid; idx < ne * 6 * Np; idx += kAdjThreads) {
    const int e = idx / (6 * Np), r = idx - e * 6 * Np, c = r / Np;
    const int64_t gi = (int64_t)e0 * 6 * Np + idx;
    const Real mu = rho[gi] + Bi * lam[gi];
    const Real s = c < 3 ? A.mat[(e0 + e) * 3 + 0] : -A.mat[(e0 + e) * 3 + 1];
    (&a[0][0][0])[idx] = mu * s;
  }
  __syncthreads();
  constexpr int NFP = (NF + 3) & ~3;
  const Real* LIFTN = A.adj_ops + 3 * Np * NpP;   // LIFT [Np][NFP]: consecutive fm adjacent
  Real* G = A.G + (int64_t)b * A.K * NF * 6;
  for (int idx = tid; idx < ne * NF; idx += kAdjThreads) {
    const int e = idx / NF, fm = idx - e * NF, f = fm / Nfp;
    const Real fsc = A.fnrm[(int64_t)(e0 + e) * 16 + f * 4 + 3];
    Real s[6] = {0, 0, 0, 0, 0, 0};
    for (int i = 0; i < Np; ++i) {
      const Real L = LIFTN[i * NFP + fm];
#pragma unroll
      for (int c = 0; c < 6; ++c) s[c] += L * a[e][c][i];
    }
    Real* go = G + ((int64_t)(e0 + e) * NF + fm) * 6;
#pragma unroll
    for (int c = 0; c < 6; ++c) go[c] = fsc * s[c];
  }
}

// ---------------------------------------------------------------- adj_main
template <typename Real, int N, bool PML, int QC = 0>
struct AdjTile {
  using D = AD<N, QC>;
  static constexpr int C = PML ? 12 : 6;
  // MU, QF, ADJ [C][Np]; FLH [NF][3]; (PML) ZZ [NqP][12]; GE, metric [16]
  static constexpr int per = 3 * C * D::Np + 3 * D::NF + (PML ? 12 * D::NqP : 0) + 16 + 16;
  static constexpr int budget = 80 * 1024;
  static constexpr int t0 = budget / (per * (int)sizeof(Real));
  static constexpr int T = t0 < 1 ? 1 : (t0 > 8 ? 8 : t0);
  static constexpr size_t smem = (size_t)T * per * sizeof(Real) + 64 * sizeof(int);
};

template <typename Real>
__device__ __forceinline__ void atomic_add_real(Real* p, Real v) {
  atomicAdd(p, v);
}

// natural logarithm: the hardware approximation in FP32 (about 1e-6
// relative error, below the FP32 adjoint's own), the library's in FP64
__device__ __forceinline__ float log_fast(float x) { return __logf(x); }
__device__ __forceinline__ double log_fast(double x) { return log(x); }

template <typename Real, int N, bool PML, int QC = 0>
__global__ void __launch_bounds__(kAdjThreads) adj_main_kernel(const AdjParams<Real> A) {
  using D = AD<N, QC>;
  constexpr int Np = D::Np, Nfp = D::Nfp, NF = D::NF, Nq = D::Nq, NpP = D::NpP, NqP = D::NqP;
  using TL = AdjTile<Real, N, PML, QC>;
  constexpr int T = TL::T, C = TL::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* MU = reinterpret_cast<Real*>(smem_raw);   // [T][C][Np]
  Real* QF = MU + T * C * Np;                      // [T][C][Np]  stage input state
  Real* ADJ = QF + T * C * Np;                     // [T][C][Np]  L^T mu
  Real* FLH = ADJ + T * C * Np;                    // [T][NF][3]  Fscale * forward flux (E rows)
  Real* ZZ = FLH + T * NF * 3;                     // [T][NqP][12] (PML)
  Real* GE = ZZ + (PML ? T * 12 * NqP : 0);        // [T] dJ/deps_k
  Real* MET = GE + T * 16;                         // [T][9] metric r_x .. t_z
  int* srcl = reinterpret_cast<int*>(MET + T * 16);
  __shared__ int nsl;
  __shared__ double red[6][kAdjThreads / 32];

  constexpr int NFP = (NF + 3) & ~3;
  const Real* DrT = A.ops;                 // D^T [Np][NpP]: DrT[j][i] = D_r[i][j]
  const Real* DsT = DrT + Np * NpP;
  const Real* DtT = DsT + Np * NpP;
  const Real* LIFTT = DtT + Np * NpP;      // [NF][NpP]
  const Real* VqT = LIFTT + NF * NpP;      // [Np][NqP]: VqT[i][q] = V_q[q][i]
  // the same operators with the other index contiguous, so that threads over
  // nodes or points read consecutive entries
  const Real* DrN = A.adj_ops;             // [Np][NpP]: DrN[j][i] = D_r[j][i]
  const Real* DsN = DrN + Np * NpP;
  const Real* DtN = DsN + Np * NpP;
  const Real* PqN = DtN + Np * NpP + Np * NFP;   // [Np][NqP]: PqN[i][q] = P_q[i][q]
  const Real* VqR = PqN + Np * NqP;              // [Nq][NpP]: VqR[q][j] = V_q[q][j]
  const unsigned char* Fmask = A.tabs;
  const unsigned char* fperm = A.tabs + NF;
  const unsigned char* fmap = A.tabs + NF + 4 * 24 * Nfp;

  const int tid = threadIdx.x, b = blockIdx.y;
  const int t0 = blockIdx.x * T;
  if (t0 >= A.n_elem) return;
  const int ne = min(T, A.n_elem - t0);
  const int eg0 = A.e_begin + t0;
  const int ep0 = eg0 - A.K0;
  const Real Bi = A.rk_b_r, Ai = A.rk_a_r, dt = A.dt_r;
  const double tst = A.t;
  Real* lam = A.lam_q + (int64_t)b * A.strideQ;
  Real* rho = A.rho_q + (int64_t)b * A.strideQ;
  const Real* qin = A.q_in + (int64_t)b * A.strideQ;
  const Real* Gb = A.G + (int64_t)b * A.K * NF * 6;

  // ---- load mu, stage input, clear accumulators
  if (tid == 0) nsl = 0;
  for (int idx = tid; idx < ne * 6 * Np; idx += kAdjThreads) {
    const int e = idx / (6 * Np), r = idx - e * 6 * Np;
    const int64_t gi = (int64_t)eg0 * 6 * Np + idx;
    MU[e * C * Np + r] = rho[gi] + Bi * lam[gi];
    QF[e * C * Np + r] = qin[gi];
  }
  if (PML) {
    const Real* lp = A.lam_p + (int64_t)b * A.strideP;
    const Real* rp = A.rho_p + (int64_t)b * A.strideP;
    const Real* pin = A.p_in + (int64_t)b * A.strideP;
    for (int idx = tid; idx < ne * 6 * Np; idx += kAdjThreads) {
      const int e = idx / (6 * Np), r = idx - e * 6 * Np;
      const int64_t gi = (int64_t)ep0 * 6 * Np + idx;
      MU[e * C * Np + 6 * Np + r] = rp[gi] + Bi * lp[gi];
      QF[e * C * Np + 6 * Np + r] = pin[gi];
    }
  }
  for (int idx = tid; idx < T * C * Np; idx += kAdjThreads) ADJ[idx] = 0;
  for (int idx = tid; idx < T; idx += kAdjThreads) GE[idx] = 0;
  for (int idx = tid; idx < ne * 9; idx += kAdjThreads)
    MET[idx] = (Real)A.geo[(int64_t)eg0 * 9 + idx];   // rounded once per element
  __syncthreads();
  for (int s = tid; s < A.nsrc; s += kAdjThreads) {
    const SrcDev& sd = A.src[s];
    if (sd.batch == b && sd.elem >= eg0 && sd.elem < eg0 + ne) {
      const int slot = atomicAdd(&nsl, 1);
      if (slot < 64) srcl[slot] = s;
    }
  }

  // ---- traces: forward flux (for dJ/deps) and the transposed flux
  for (int idx = tid; idx < ne * NF; idx += kAdjThreads) {
    const int e = idx / NF, fm = idx - e * NF, f = fm / Nfp, m = fm - f * Nfp;
    const int eg = eg0 + e;
    const int ni = Fmask[fm];
    const Real* nf = A.fnrm + (int64_t)eg * 16 + f * 4;
    const Real n[3] = {nf[0], nf[1], nf[2]}, fsc = nf[3];
    const Real* qf = QF + e * C * Np;
    Real Em[3], Hm[3], Ep[3], Hp[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) { Em[c] = qf[c * Np + ni]; Hm[c] = qf[(3 + c) * Np + ni]; }
    const Real ZM = A.mat[eg * 3 + 2];
    const int nb = A.nbr[eg * 4 + f];
    Real ZP = ZM;
    const Real* go = Gb + ((int64_t)eg * NF + fm) * 6;
    Real gH[3] = {go[0], go[1], go[2]}, gE[3] = {go[3], go[4], go[5]};
    Real gH2[3] = {0, 0, 0}, gE2[3] = {0, 0, 0};
    if (nb >= 0) {
      const int code = A.code[eg * 4 + f];
      const int np2 = fperm[(f * 24 + code) * Nfp + m];
      const int fm2 = (code / 6) * Nfp + fmap[(f * 24 + code) * Nfp + m];
      const Real* qn = qin + (int64_t)nb * 6 * Np + np2;
#pragma unroll
      for (int c = 0; c < 3; ++c) { Ep[c] = qn[c * Np]; Hp[c] = qn[(3 + c) * Np]; }
      ZP = A.mat[nb * 3 + 2];
      const Real* g2 = Gb + ((int64_t)nb * NF + fm2) * 6;
#pragma unroll
      for (int c = 0; c < 3; ++c) { gH2[c] = g2[c]; gE2[c] = g2[3 + c]; }
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c) { Ep[c] = -Em[c]; Hp[c] = Hm[c]; }
    }
    const Real al = A.alpha_r;
    const Real YM = Real(1) / ZM, YP = Real(1) / ZP;
    const Real sH = Real(1) / (ZM + ZP), sE = Real(1) / (YM + YP);
    Real dE[3], dH[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) { dE[c] = Ep[c] - Em[c]; dH[c] = Hp[c] - Hm[c]; }
    const Real ndE = n[0] * dE[0] + n[1] * dE[1] + n[2] * dE[2];
    const Real ndH = n[0] * dH[0] + n[1] * dH[1] + n[2] * dH[2];
    Real nxdH[3], nxdE[3];
    cross3(n, dH, nxdH);
    cross3(n, dE, nxdE);
    Real fCH[3], fCE[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      fCH[c] = sH * (ZP * nxdH[c] - al * (n[c] * ndE - dE[c]));
      fCE[c] = sE * (YP * nxdE[c] + al * (n[c] * ndH - dH[c]));
      FLH[(e * NF + fm) * 3 + c] = fsc * fCH[c];
    }
    // transpose of the own flux with respect to dE, dH
    Real nxgH[3], nxgE[3];
    cross3(n, gH, nxgH);
    cross3(n, gE, nxgE);
    const Real ngH = n[0] * gH[0] + n[1] * gH[1] + n[2] * gH[2];
    const Real ngE = n[0] * gE[0] + n[1] * gE[1] + n[2] * gE[2];
    Real adE[3], adH[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      adH[c] = -sH * ZP * nxgH[c] + sE * al * (n[c] * ngE - gE[c]);
      adE[c] = -sH * al * (n[c] * ngH - gH[c]) - sE * YP * nxgE[c];
    }
    Real* ad = ADJ + e * C * Np;
    // impedance derivative of eps_k: dZ/deps = -Z/(2 eps), dY/deps = Y/(2 eps)
    const Real ie = A.mat[eg * 3 + 0];
    const Real dZ = -ZM * ie * Real(0.5), dY = YM * ie * Real(0.5);
    Real ge = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      ge += gH[c] * (-fCH[c] * sH) * dZ + gE[c] * (-fCE[c] * sE) * dY;   // Z-, Y- of k
    }
    if (nb >= 0) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        atomic_add_real(&ad[c * Np + ni], -adE[c]);
        atomic_add_real(&ad[(3 + c) * Np + ni], -adH[c]);
      }
      // the neighbour's flux at the same point: normal -n, jumps -dE, -dH,
      // its Z- is Z_nb and its Z+ is Z_k
      Real nxg2H[3], nxg2E[3];
      cross3(n, gH2, nxg2H);
      cross3(n, gE2, nxg2E);
      const Real ng2H = n[0] * gH2[0] + n[1] * gH2[1] + n[2] * gH2[2];
      const Real ng2E = n[0] * gE2[0] + n[1] * gE2[1] + n[2] * gE2[2];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const Real a2H = sH * ZM * nxg2H[c] + sE * al * (n[c] * ng2E - gE2[c]);
        const Real a2E = -sH * al * (n[c] * ng2H - gH2[c]) + sE * YM * nxg2E[c];
        atomic_add_real(&ad[c * Np + ni], a2E);
        atomic_add_real(&ad[(3 + c) * Np + ni], a2H);
        const Real fCH2 = sH * (ZM * nxdH[c] + al * (n[c] * ndE - dE[c]));
        const Real fCE2 = sE * (YM * nxdE[c] - al * (n[c] * ndH - dH[c]));
        ge += gH2[c] * (sH * nxdH[c] - fCH2 * sH) * dZ + gE2[c] * (sE * nxdE[c] - fCE2 * sE) * dY;
      }
    } else {
      // perfect electric conductor: E+ = -E-, H+ = H-  (dE = -2E-, dH = 0), Z+ = Z-
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        atomic_add_real(&ad[c * Np + ni], Real(-2) * adE[c]);
        ge += gH[c] * (sH * nxdH[c] - fCH[c] * sH) * dZ + gE[c] * (sE * nxdE[c] - fCE[c] * sE) * dY;
      }
    }
    atomic_add_real(&GE[e], ge);
  }
  __syncthreads();
  const int nsrc_l = min(nsl, 64);

  // ---- volume: curl^T of (mu_E/eps, -mu_H/mu); forward Cbar(H) for dJ/deps
  for (int idx = tid; idx < ne * Np; idx += kAdjThreads) {
    const int e = idx / Np, i = idx - e * Np;
    const int eg = eg0 + e;
    const Real ie = A.mat[eg * 3 + 0], im = A.mat[eg * 3 + 1];
    const Real* mu = MU + e * C * Np;
    const Real* qf = QF + e * C * Np;
    Real tr[6][3];   // (D_r^T a_c, D_s^T a_c, D_t^T a_c) at node i, a = (mu_E/eps, -mu_H/mu)
    Real fw[3][3];   // forward d/dr, d/ds, d/dt of H at node i
#pragma unroll
    for (int c = 0; c < 6; ++c) tr[c][0] = tr[c][1] = tr[c][2] = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) fw[c][0] = fw[c][1] = fw[c][2] = 0;
    for (int j = 0; j < Np; ++j) {
      const Real r1 = DrN[j * NpP + i], s1 = DsN[j * NpP + i], t1 = DtN[j * NpP + i];  // D[j][i]
      const Real r2 = DrT[j * NpP + i], s2 = DsT[j * NpP + i], t2 = DtT[j * NpP + i];  // D[i][j]
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        const Real a = c < 3 ? mu[c * Np + j] * ie : -mu[c * Np + j] * im;
        tr[c][0] += r1 * a; tr[c][1] += s1 * a; tr[c][2] += t1 * a;
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const Real h = qf[(3 + c) * Np + j];
        fw[c][0] += r2 * h; fw[c][1] += s2 * h; fw[c][2] += t2 * h;
      }
    }
    const Real* gd = MET + e * 9;
    const Real rx = gd[0], ry = gd[1], rz = gd[2];
    const Real sx = gd[3], sy = gd[4], sz = gd[5];
    const Real tx = gd[6], ty = gd[7], tz = gd[8];
    // dT_x a = r_x D_r^T a + s_x D_s^T a + t_x D_t^T a (constant metric)
    Real dtx[6], dty[6], dtz[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      dtx[c] = rx * tr[c][0] + sx * tr[c][1] + tx * tr[c][2];
      dty[c] = ry * tr[c][0] + sy * tr[c][1] + ty * tr[c][2];
      dtz[c] = rz * tr[c][0] + sz * tr[c][1] + tz * tr[c][2];
    }
    Real* ad = ADJ + e * C * Np;
    // curl^T a: F0 += dz^T a1 - dy^T a2, F1 += dx^T a2 - dz^T a0, F2 += dy^T a0 - dx^T a1
    // a_E (from the E rows) acts on H, a_H (from the H rows) acts on E
    ad[3 * Np + i] += dtz[1] - dty[2];
    ad[4 * Np + i] += dtx[2] - dtz[0];
    ad[5 * Np + i] += dty[0] - dtx[1];
    ad[0 * Np + i] += dtz[4] - dty[5];
    ad[1 * Np + i] += dtx[5] - dtz[3];
    ad[2 * Np + i] += dty[3] - dtx[4];
    // forward Cbar(H) at node i (curl H + LIFT flux - source)
    Real hx[3], hy[3], hz[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      hx[c] = rx * fw[c][0] + sx * fw[c][1] + tx * fw[c][2];
      hy[c] = ry * fw[c][0] + sy * fw[c][1] + ty * fw[c][2];
      hz[c] = rz * fw[c][0] + sz * fw[c][1] + tz * fw[c][2];
    }
    Real CH[3] = {hy[2] - hz[1], hz[0] - hx[2], hx[1] - hy[0]};
    for (int fm = 0; fm < NF; ++fm) {
      const Real L = LIFTT[fm * NpP + i];
#pragma unroll
      for (int c = 0; c < 3; ++c) CH[c] += L * FLH[(e * NF + fm) * 3 + c];
    }
    for (int s = 0; s < nsrc_l; ++s) {
      const SrcDev& sd = A.src[srcl[s]];
      if (sd.elem != eg) continue;
      const double tau = sd.width;
      const double g = exp(-(tst - sd.t0) * (tst - sd.t0) / (4.0 * tau * tau));
      const Real jt = (Real)(sd.amp * (-(tst - sd.t0) / (2.0 * tau * tau)) * g);
      const Real w = A.src_w[srcl[s] * Np + i];
#pragma unroll
      for (int c = 0; c < 3; ++c) CH[c] -= jt * (Real)sd.dir[c] * w;
    }
    // d/deps_k of mu_E . Cbar(H)/eps_k = -mu_E . Cbar(H) / eps_k^2
    Real ge = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) ge -= mu[c * Np + i] * CH[c] * ie * ie;
    atomic_add_real(&GE[e], ge);
  }

  Real gp[6] = {0, 0, 0, 0, 0, 0};   // d/dsigma_max[3], d/dp_sigma[3] (this thread's points)
  if (PML) {
    __syncthreads();
    // ---- quadrature points: w = P_q^T mu, forward v = V_q q_in, the pullback
    //      values of eqs. 26-29 transposed, and the profile derivatives.  Each
    //      thread takes QB points of one element and one field group (g = 0:
    //      E with P^E, g = 1: H with P^H; eq. 9 and the derivative sums never
    //      mix the groups), so every mu and q_in value it loads serves QB
    //      points.  ZZ[e][q][g][k]: k < 3 the field row, k >= 3 the P row.
    constexpr int QB = Nq >= 48 ? 4 : 2;
    constexpr int NQB = (Nq + QB - 1) / QB;
    constexpr int NQI = NQB * 2;   // items per element (even: partner items on lanes 2m, 2m + 1)
    const Real ie0 = A.inv_eps0_r;
    const Real* rsm = A.inv_sigma_max;   // 1 / sigma_max, 1 / p_sigma per axis (0: unset)
    const Real* rps = A.inv_p_sigma;
    // every lane runs the same number of iterations: the E and H items of a
    // point sit on neighbouring lanes and add their derivative shares by a
    // shuffle before the per-point scaling
    for (int base = 0; base < ne * NQI; base += kAdjThreads) {
      const int idx = base + tid;
      const bool act = idx < ne * NQI;
      const int e = act ? idx / NQI : 0, r = act ? idx - e * NQI : 0;
      const int g = r & 1, q0 = (r >> 1) * QB;
      const Real* mu = MU + e * C * Np;
      const Real* qf = QF + e * C * Np;
      Real w[QB][6], v[QB][6];
#pragma unroll
      for (int k = 0; k < QB; ++k)
#pragma unroll
        for (int c = 0; c < 6; ++c) { w[k][c] = 0; v[k][c] = 0; }
      if (act) {
        for (int i = 0; i < Np; ++i) {
          Real m[6], f[6];
#pragma unroll
          for (int u = 0; u < 3; ++u) {
            m[u] = mu[(3 * g + u) * Np + i];
            m[3 + u] = mu[(6 + 3 * g + u) * Np + i];
            f[u] = qf[(3 * g + u) * Np + i];
            f[3 + u] = qf[(6 + 3 * g + u) * Np + i];
          }
#pragma unroll
          for (int k = 0; k < QB; ++k) {
            const int q = q0 + k;   // < NqP: the padded columns hold zeros
            const Real pq = PqN[i * NqP + q];   // P_q[i][q]
            const Real vq = VqT[i * NqP + q];   // V_q[q][i]
#pragma unroll
            for (int c = 0; c < 6; ++c) {
              w[k][c] += pq * m[c];
              v[k][c] += vq * f[c];
            }
          }
        }
      }
#pragma unroll
      for (int k = 0; k < QB; ++k) {
        const int q = q0 + k;
        const bool live = act && q < Nq;
        Real sg[3] = {0, 0, 0};
        if (live) {
          const int64_t sb = (int64_t)(ep0 + e) * 3 * NqP + q;
          sg[0] = A.sig[sb];
          sg[1] = A.sig[sb + NqP];
          sg[2] = A.sig[sb + 2 * NqP];
          Real* zz = ZZ + ((e * NqP + q) * 2 + g) * 6;
#pragma unroll
          for (int u = 0; u < 3; ++u) {
            const int vv = (u + 1) % 3, ww = (u + 2) % 3;
            const Real bu = (sg[vv] + sg[ww] - sg[u]) * ie0;
            const Real cu = sg[vv] * sg[ww] * ie0 * ie0 - bu * sg[u] * ie0;
            const Real du = sg[u] * ie0;
            zz[u] = -bu * w[k][u] + w[k][3 + u];
            zz[3 + u] = -cu * w[k][u] - du * w[k][3 + u];
          }
        }
        // d/dtheta of mu . f through b, c, d at this point.  It is linear in
        // the derivative of sigma_a: one sum per axis with d sigma_a = 1 (this
        // group's share, then both groups'), scaled by d sigma_a / d
        // sigma_max_a = sigma_a / sigma_max_a and d sigma_a / d p_a =
        // sigma_a log(sigma_a / sigma_max_a) / p_a
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          Real acc = 0;
          if (live && sg[a] > 0) {
#pragma unroll
            for (int u = 0; u < 3; ++u) {
              const int vv = (u + 1) % 3, ww = (u + 2) % 3;
              const Real ds_u = u == a ? Real(1) : Real(0), ds_v = vv == a ? Real(1) : Real(0);
              const Real ds_w = ww == a ? Real(1) : Real(0);
              const Real bu = (sg[vv] + sg[ww] - sg[u]) * ie0;
              const Real db = (ds_v + ds_w - ds_u) * ie0;
              const Real dc =
                  (ds_v * sg[ww] + sg[vv] * ds_w) * ie0 * ie0 - (db * sg[u] + bu * ds_u) * ie0;
              const Real dd = ds_u * ie0;
              acc -= w[k][u] * (db * v[k][u] + dc * v[k][3 + u]) + dd * w[k][3 + u] * v[k][3 + u];
            }
          }
          acc += __shfl_xor_sync(0xffffffffu, acc, 1);
          if (g == 0 && live && sg[a] > 0 && rsm[a] > 0) {
            const Real x = sg[a] * rsm[a];
            gp[a] += x * acc;
            gp[3 + a] += sg[a] * log_fast(x) * rps[a] * acc;
          }
        }
      }
    }
    __syncthreads();
    // ---- V_q^T pullback to the nodes: two nodes of one element and one
    //      field group per thread
    constexpr int JB = 2;
    constexpr int NJB = (Np + JB - 1) / JB;
    for (int idx = tid; idx < ne * NJB * 2; idx += kAdjThreads) {
      const int e = idx / (NJB * 2), r = idx - e * (NJB * 2), g = r & 1, j0 = (r >> 1) * JB;
      Real sacc[JB][6];
#pragma unroll
      for (int k = 0; k < JB; ++k)
#pragma unroll
        for (int c = 0; c < 6; ++c) sacc[k][c] = 0;
      for (int q = 0; q < Nq; ++q) {
        const Real* zz = ZZ + ((e * NqP + q) * 2 + g) * 6;
        Real z[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) z[c] = zz[c];
#pragma unroll
        for (int k = 0; k < JB; ++k) {
          const int j = j0 + k;   // < NpP: the padded columns hold zeros
          const Real vq = VqR[q * NpP + j];   // V_q[q][j]
#pragma unroll
          for (int c = 0; c < 6; ++c) sacc[k][c] += vq * z[c];
        }
      }
      Real* ad = ADJ + e * C * Np;
#pragma unroll
      for (int k = 0; k < JB; ++k) {
        const int j = j0 + k;
        if (j >= Np) break;
#pragma unroll
        for (int u = 0; u < 3; ++u) {
          ad[(3 * g + u) * Np + j] += sacc[k][u];
          ad[(6 + 3 * g + u) * Np + j] += sacc[k][3 + u];
        }
      }
    }
  }
  __syncthreads();

  // ---- lambda_in = lambda_out + dt L^T mu, rho_prev = A_i mu; dJ/deps_k
  for (int idx = tid; idx < ne * 6 * Np; idx += kAdjThreads) {
    const int e = idx / (6 * Np), r = idx - e * 6 * Np;
    const int64_t gi = (int64_t)eg0 * 6 * Np + idx;
    lam[gi] = lam[gi] + dt * ADJ[e * C * Np + r];
    rho[gi] = Ai * MU[e * C * Np + r];
  }
  if (PML) {
    Real* lp = A.lam_p + (int64_t)b * A.strideP;
    Real* rp = A.rho_p + (int64_t)b * A.strideP;
    for (int idx = tid; idx < ne * 6 * Np; idx += kAdjThreads) {
      const int e = idx / (6 * Np), r = idx - e * 6 * Np;
      const int64_t gi = (int64_t)ep0 * 6 * Np + idx;
      lp[gi] = lp[gi] + dt * ADJ[e * C * Np + 6 * Np + r];
      rp[gi] = Ai * MU[e * C * Np + 6 * Np + r];
    }
  }
  for (int e = tid; e < ne; e += kAdjThreads)
    A.grad_eps[(int64_t)b * A.K + eg0 + e] += (double)dt * (double)GE[e];
  if (PML) {
    // block reduction of the profile derivatives: across the warp in the
    // working precision, across warps in double
    const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      Real v = gp[k];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[k][wid] = (double)v;
    }
    __syncthreads();
    if (tid < 6) {
      double s = 0;
      for (int w = 0; w < kAdjThreads / 32; ++w) s += red[tid][w];
      atomicAdd(&A.grad_prof[b * 6 + tid], (double)dt * s);
    }
  }
}

// lambda_E += dJ/dE = 2 (l . E) l at each probe, from the step-end state
template <typename Real>
__global__ void adj_probe_kernel(const Real* q, int64_t strideQ, int nprobe, int nb, int Np,
                                 const int* elem, const double* ell, Real* lam) {
  const int p = blockIdx.x, b = blockIdx.y, lane = threadIdx.x;
  const Real* qe = q + (int64_t)b * strideQ + (int64_t)elem[p] * 6 * Np;
  double e3[3] = {0, 0, 0};
  for (int i = lane; i < Np; i += 32)
    for (int c = 0; c < 3; ++c) e3[c] += ell[(int64_t)p * Np + i] * (double)qe[c * Np + i];
  for (int c = 0; c < 3; ++c)
    for (int o = 16; o > 0; o >>= 1) e3[c] += __shfl_xor_sync(0xffffffffu, e3[c], o);
  Real* le = lam + (int64_t)b * strideQ + (int64_t)elem[p] * 6 * Np;
  for (int i = lane; i < Np; i += 32)
    for (int c = 0; c < 3; ++c)
      atomicAdd(&le[c * Np + i], (Real)(2.0 * e3[c] * ell[(int64_t)p * Np + i]));
}

template <typename Real, int N>
cudaError_t adj_stage_n(const AdjParams<Real>& P, int nb, cudaStream_t s, int qc) {
  {
    dim3 g((P.K + 7) / 8, nb);
    adj_lift_kernel<Real, N><<<g, kAdjThreads, 0, s>>>(P);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  // non-PML elements, then PML elements
  for (int cls = 0; cls < 2; ++cls) {
    AdjParams<Real> Q = P;
    Q.e_begin = cls == 0 ? 0 : P.K0;
    Q.n_elem = cls == 0 ? P.K0 : P.K - P.K0;
    if (Q.n_elem <= 0) continue;
    if (cls == 0) {
      using TL = AdjTile<Real, N, false>;
      dim3 g((Q.n_elem + TL::T - 1) / TL::T, nb);
      adj_main_kernel<Real, N, false><<<g, kAdjThreads, TL::smem, s>>>(Q);
    } else if (qc) {
      using TL = AdjTile<Real, N, true, 1>;
      dim3 g((Q.n_elem + TL::T - 1) / TL::T, nb);
      adj_main_kernel<Real, N, true, 1><<<g, kAdjThreads, TL::smem, s>>>(Q);
    } else {
      using TL = AdjTile<Real, N, true>;
      dim3 g((Q.n_elem + TL::T - 1) / TL::T, nb);
      adj_main_kernel<Real, N, true><<<g, kAdjThreads, TL::smem, s>>>(Q);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename Real, int N>
cudaError_t adj_configure_n() {
  cudaError_t e = cudaFuncSetAttribute(adj_main_kernel<Real, N, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)AdjTile<Real, N, false>::smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(adj_main_kernel<Real, N, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)AdjTile<Real, N, true>::smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(adj_main_kernel<Real, N, true, 1>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)AdjTile<Real, N, true, 1>::smem);
  return e;
}

}  // namespace

template <typename Real>
cudaError_t configure_adjoint_kernels(int N) {
  switch (N) {
    case 1: return adj_configure_n<Real, 1>();
    case 2: return adj_configure_n<Real, 2>();
    case 3: return adj_configure_n<Real, 3>();
    case 4: return adj_configure_n<Real, 4>();
    case 5: return adj_configure_n<Real, 5>();
    default: return cudaErrorInvalidValue;
  }
}
template cudaError_t configure_adjoint_kernels<double>(int);
template cudaError_t configure_adjoint_kernels<float>(int);

template <typename Real>
cudaError_t launch_adjoint_stage(int N, const AdjParams<Real>& P, int nb, cudaStream_t s,
                                 int qc) {
  switch (N) {
    case 1: return adj_stage_n<Real, 1>(P, nb, s, qc);
    case 2: return adj_stage_n<Real, 2>(P, nb, s, qc);
    case 3: return adj_stage_n<Real, 3>(P, nb, s, qc);
    case 4: return adj_stage_n<Real, 4>(P, nb, s, qc);
    case 5: return adj_stage_n<Real, 5>(P, nb, s, qc);
    default: return cudaErrorInvalidValue;
  }
}
template cudaError_t launch_adjoint_stage<double>(int, const AdjParams<double>&, int, cudaStream_t,
                                                  int);
template cudaError_t launch_adjoint_stage<float>(int, const AdjParams<float>&, int, cudaStream_t,
                                                 int);

template <typename Real>
cudaError_t launch_adjoint_probes(const Real* q, int64_t strideQ, int nprobe, int nb, int Np,
                                  const int* elem, const double* ell, Real* lam, cudaStream_t s) {
  if (nprobe <= 0) return cudaSuccess;
  adj_probe_kernel<Real><<<dim3(nprobe, nb), 32, 0, s>>>(q, strideQ, nprobe, nb, Np, elem, ell, lam);
  return cudaGetLastError();
}
template cudaError_t launch_adjoint_probes<double>(const double*, int64_t, int, int, int, const int*,
                                                   const double*, double*, cudaStream_t);
template cudaError_t launch_adjoint_probes<float>(const float*, int64_t, int, int, int, const int*,
                                                  const double*, float*, cudaStream_t);

}  // namespace wadg
