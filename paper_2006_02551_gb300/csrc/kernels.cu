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

#include <algorithm>
#include <cstdio>
#include <type_traits>

namespace wadg {

template <int N>
struct Dims {
  static constexpr int Np = (N + 1) * (N + 2) * (N + 3) / 6;
  static constexpr int Nfp = (N + 1) * (N + 2) / 2;
  static constexpr int Nq = (N + 1) * (N + 1) * (N + 1);
  static constexpr int NF = 4 * Nfp;
  static constexpr int NpP = (Np + 3) & ~3;   // padded to whole quads
  static constexpr int NqP = (Nq + 3) & ~3;
  static constexpr int NIQ = NpP / 4;         // node quads
  static constexpr int NQQ = NqP / 4;         // quadrature-point quads
};

// Launch configuration: persistent blocks, the reference operators staged in
// shared memory once per block, tiles of T elements processed in a loop.
template <typename Real, int N, bool PML, int NT_ = 0>
struct Tile {
  using D = Dims<N>;
  // threads of a block: the single-class launches use 512 for FP32 PML tiles;
  // the grouped launch fixes 256 for every class
  static constexpr int THREADS = NT_ > 0 ? NT_ : ((sizeof(Real) == 4 && PML) ? 512 : 256);
  static constexpr int CF = PML ? 12 : 6;                  // field components held
  static constexpr int f_sz = D::Np * CF;                  // F[e][j][CF]
  static constexpr int u_sz = PML ? ((D::NF * 6 > D::NqP * 12) ? D::NF * 6 : D::NqP * 12)
                                  : D::NF * 6;             // flux[e][f][6] / tz[e][q][12]
  static constexpr int r_sz = PML ? D::NpP * 6 : 0;        // rs[e][i][6]
  static constexpr int per_elem = f_sz + u_sz + r_sz + 16 + 12;
  // operators: DrT DsT DtT [Np][NpP], LIFTT [NF][NpP] (+ VqT [Np][NqP], PqT [Nq][NpP]);
  // staged in shared memory when they fit, read through L1 otherwise
  static constexpr int ops_all = 3 * D::Np * D::NpP + D::NF * D::NpP +
                                 (PML ? D::Np * D::NqP + D::Nq * D::NpP : 0);
  static constexpr bool OPS_SMEM = ops_all * (int)sizeof(Real) <= 160 * 1024;
  static constexpr int ops_sz = OPS_SMEM ? ops_all : 0;
  static constexpr int budget = (PML || sizeof(Real) == 8) ? 200 * 1024 : 100 * 1024;
  static constexpr int avail = budget - ops_sz * (int)sizeof(Real) - 256;
  static constexpr int t0 = avail / (per_elem * (int)sizeof(Real));
  // enough tiles of work per phase for the block's threads, not more
  static constexpr int t_tasks = PML ? THREADS / D::NQQ : THREADS / (2 * D::NIQ);
  static constexpr int t1 = t0 < t_tasks ? t0 : t_tasks;
  static constexpr int T = t1 < 1 ? 1 : (t1 > 32 ? 32 : t1);
  static constexpr size_t smem =
      (size_t)(ops_sz + T * per_elem) * sizeof(Real) + 64 * sizeof(int);
};

__device__ __forceinline__ double dipole_current(const SrcDev& s, double t) {
  double tau = s.width;
  double g = exp(-(t - s.t0) * (t - s.t0) / (4.0 * tau * tau));
  return s.amp * (-(t - s.t0) / (2.0 * tau * tau)) * g;
}

// global read-only loads of four consecutive values (16-byte aligned)
__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
  float4 t = __ldg(reinterpret_cast<const float4*>(p));
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&v)[4]) {
  double2 a = __ldg(reinterpret_cast<const double2*>(p));
  double2 b = __ldg(reinterpret_cast<const double2*>(p + 2));
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
// shared-memory vector loads
__device__ __forceinline__ void lds4(const float* p, float* v) {
  float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void lds4(const double* p, double* v) {
  double2 a = *reinterpret_cast<const double2*>(p);
  double2 b = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void sts4(float* p, const float* v) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void sts4(double* p, const double* v) {
  *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
}
__device__ __forceinline__ void lds2(const float* p, float* v) {
  float2 t = *reinterpret_cast<const float2*>(p);
  v[0] = t.x; v[1] = t.y;
}
__device__ __forceinline__ void lds2(const double* p, double* v) {
  double2 t = *reinterpret_cast<const double2*>(p);
  v[0] = t.x; v[1] = t.y;
}

// Stage kernel.  Threads work on register tiles: 4 nodes x 3 components x 3
// reference derivatives (curl), 4 quadrature points x 12 components (V_q),
// 4 nodes x 4 components (P_q).  All operator reads come from shared memory.
// Body of the stage kernel for one element class of one context; smem_raw is
// the block's dynamic shared memory.  Static schedule: block `bid` of `nblk`
// takes tiles bid, bid + nblk, ...  Dynamic schedule (dyn != nullptr, the
// grouped launch): the block takes tiles from the counter *dyn until they run
// out.
template <typename Real, int N, bool PML, bool KAPPA, bool STORED, int NT_>
__device__ __forceinline__ void stage_body(const StageParams<Real>& P, unsigned char* smem_raw,
                                           int bid, int nblk, int* dyn = nullptr) {
  using D = Dims<N>;
  constexpr int Np = D::Np, Nfp = D::Nfp, Nq = D::Nq, NF = D::NF;
  constexpr int NpP = D::NpP, NqP = D::NqP, NIQ = D::NIQ, NQQ = D::NQQ;
  using TL = Tile<Real, N, PML, NT_>;
  constexpr int T = TL::T, CF = TL::CF, NT = TL::THREADS;
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  const Real* DrT = TL::OPS_SMEM ? sm : P.ops;   // operators
  const Real* DsT = DrT + Np * NpP;
  const Real* DtT = DsT + Np * NpP;
  const Real* LIFTT = DtT + Np * NpP;
  const Real* VqT = LIFTT + NF * NpP;   // PML only
  const Real* PqT = VqT + Np * NqP;     // PML only
  // elements per tile: T, or fewer when the launch asks for smaller tiles
  // (the shared-memory carve-up follows, so smaller tiles need less of it)
  const int TE = P.tile_elems > 0 && P.tile_elems < T ? P.tile_elems : T;
  Real* F = sm + TL::ops_sz;         // [TE][Np][CF]
  Real* U = F + TE * TL::f_sz;       // flux [TE][NF][6] | tz [TE][NqP][12]
  Real* RS = U + TE * TL::u_sz;      // [TE][NpP][6]
  Real* nrm = RS + TE * TL::r_sz;    // [TE][4][4]
  Real* met = nrm + TE * 16;         // [TE][12] (9 used)
  int* srcl = reinterpret_cast<int*>(met + TE * 12);
  __shared__ int nsl;

  const unsigned char* Fmask = P.tabs;
  const unsigned char* fperm = P.tabs + NF;
  const int tid = threadIdx.x;

  // operators -> shared memory, once per block
  for (int idx = tid; idx < TL::ops_sz / 2; idx += NT) {
    const Real* src = P.ops + 2 * idx;
    sm[2 * idx] = src[0];
    sm[2 * idx + 1] = src[1];
  }
  if ((TL::ops_sz & 1) && tid == 0) sm[TL::ops_sz - 1] = P.ops[TL::ops_sz - 1];

  const double tbase = P.t_dev ? *P.t_dev : P.t;
  const double tst = tbase + P.rk_c * P.dt;
  const Real rka = (Real)P.rk_a, rkb = (Real)P.rk_b, rdt = (Real)P.dt;
  const int tiles_per_batch = (P.n_elem + TE - 1) / TE;
  const int ntiles = tiles_per_batch * P.nb;

  __shared__ int dyn_tile;
  auto next_tile = [&](int cur) -> int {
    if (!dyn) return cur < 0 ? bid : cur + nblk;
    __syncthreads();   // every thread has read the previous value
    if (tid == 0) dyn_tile = atomicAdd(dyn, 1);
    __syncthreads();
    return dyn_tile;
  };
  for (int tile = next_tile(-1); tile < ntiles; tile = next_tile(tile)) {
  const int b = tile / tiles_per_batch;
  const int t0 = (tile - b * tiles_per_batch) * TE;
  const int ne = min(TE, P.n_elem - t0);
  const int eg0 = P.e_begin + t0;
  const int ep0 = eg0 - P.K0;
  const Real* qin = P.qin + (int64_t)b * P.strideQ;
  Real* qout = P.qout + (int64_t)b * P.strideQ;
  Real* resq = P.resq + (int64_t)b * P.strideQ;
  Real* pio = P.p + (int64_t)b * P.strideP;
  Real* resp = P.resp + (int64_t)b * P.strideP;
  __syncthreads();   // previous tile done with the shared buffers

  // ---- phase 0: fields (component-fastest), geometry, sources of the tile
  if (tid == 0) nsl = 0;
  for (int idx = tid; idx < ne * 6 * Np; idx += NT) {
    const int e = idx / (6 * Np), r = idx - e * 6 * Np, c = r / Np, j = r - c * Np;
    F[(e * Np + j) * CF + c] = qin[(int64_t)eg0 * 6 * Np + idx];
  }
  if (PML) {
    const Real* pin = pio + (int64_t)ep0 * 6 * Np;
    for (int idx = tid; idx < ne * 6 * Np; idx += NT) {
      const int e = idx / (6 * Np), r = idx - e * 6 * Np, c = r / Np, j = r - c * Np;
      F[(e * Np + j) * CF + 6 + c] = pin[idx];
    }
  }
  for (int idx = tid; idx < ne * 16; idx += NT)
    nrm[idx] = P.fnrm[(int64_t)eg0 * 16 + idx];   // n_x, n_y, n_z, Fscale per face
  for (int idx = tid; idx < ne * 9; idx += NT) {
    const int e = idx / 9, k = idx - e * 9;
    met[e * 12 + k] = (Real)P.geo[(int64_t)eg0 * 9 + idx];
  }
  __syncthreads();
  for (int s = tid; s < P.nsrc; s += NT) {
    const SrcDev& sd = P.src[s];
    if (sd.batch == b && sd.elem >= eg0 && sd.elem < eg0 + ne) {
      const int slot = atomicAdd(&nsl, 1);
      if (slot < 64) srcl[slot] = s;
    }
  }

  // ---- phase 1: upwind flux at the 4 Nfp trace nodes, scaled by Fscale
  Real* FL = U;   // [T][NF][6]: 0..2 drive E, 3..5 drive H
  for (int idx = tid; idx < ne * NF; idx += NT) {
    const int e = idx / NF, fm = idx - e * NF;
    const int f = fm / Nfp, m = fm - f * Nfp;
    const int eg = eg0 + e;
    const int ni = Fmask[fm];
    const Real* nn = nrm + (e * 4 + f) * 4;
    const Real nx = nn[0], ny = nn[1], nz = nn[2], fsc = nn[3];
    const Real* fe = F + (e * Np + ni) * CF;
    Real Em[3] = {fe[0], fe[1], fe[2]}, Hm[3] = {fe[3], fe[4], fe[5]};
    Real Ep[3], Hp[3];
    const Real ZM = P.mat[eg * 3 + 2];
    Real ZP = ZM;
    const int nb = P.nbr[eg * 4 + f];
    if (nb >= 0) {
      const int code = P.code[eg * 4 + f];
      const int np2 = fperm[(f * 24 + code) * Nfp + m];
      const Real* qn = qin + (int64_t)nb * 6 * Np + np2;
#pragma unroll
      for (int c = 0; c < 3; ++c) { Ep[c] = qn[c * Np]; Hp[c] = qn[(3 + c) * Np]; }
      ZP = P.mat[nb * 3 + 2];
    } else {   // perfect electric conductor: mirror state
#pragma unroll
      for (int c = 0; c < 3; ++c) { Ep[c] = -Em[c]; Hp[c] = Hm[c]; }
    }
    const Real dEx = Ep[0] - Em[0], dEy = Ep[1] - Em[1], dEz = Ep[2] - Em[2];
    const Real dHx = Hp[0] - Hm[0], dHy = Hp[1] - Hm[1], dHz = Hp[2] - Hm[2];
    const Real ndE = nx * dEx + ny * dEy + nz * dEz;
    const Real ndH = nx * dHx + ny * dHy + nz * dHz;
    const Real cHx = ny * dHz - nz * dHy, cHy = nz * dHx - nx * dHz, cHz = nx * dHy - ny * dHx;
    const Real cEx = ny * dEz - nz * dEy, cEy = nz * dEx - nx * dEz, cEz = nx * dEy - ny * dEx;
    const Real al = (Real)P.alpha;
    const Real YM = Real(1) / ZM, YP = Real(1) / ZP;
    const Real sH = fsc / (ZM + ZP), sE = fsc / (YM + YP);
    Real* fo = FL + (e * NF + fm) * 6;
    // drives E: (Z+ n x dH - alpha n x (n x dE)) / (Z- + Z+)
    fo[0] = sH * (ZP * cHx - al * (nx * ndE - dEx));
    fo[1] = sH * (ZP * cHy - al * (ny * ndE - dEy));
    fo[2] = sH * (ZP * cHz - al * (nz * ndE - dEz));
    // drives H: (Y+ n x dE + alpha n x (n x dH)) / (Y- + Y+)
    fo[3] = sE * (YP * cEx + al * (nx * ndH - dHx));
    fo[4] = sE * (YP * cEy + al * (ny * ndH - dHy));
    fo[5] = sE * (YP * cEz + al * (nz * ndH - dHz));
  }
  __syncthreads();
  const int nsrc_l = min(nsl, 64);

  // ---- phase 2 (+ phase 3 in PML tiles, same loop: they are independent)
  //   curl task (e, fld, iq): fld 0: Cbar(E) -> rhs_H = -Cbar(E)/mu,
  //                           fld 1: Cbar(H) -> rhs_E =  Cbar(H)/eps
  //   V_q task (e, qq): 12 fields at 4 quadrature points, then eq. 9 pointwise
  // In PML tiles the V_q results go to TZ, which aliases FL; so the V_q tasks
  // must not start before every curl task has read FL: they run after a
  // barrier in the second loop below.
  const int n2 = ne * 2 * NIQ;
  for (int task = tid; task < n2; task += NT) {
    const int e = task / (2 * NIQ), r = task - e * 2 * NIQ, fld = r / NIQ, iq = r - fld * NIQ;
    const int eg = eg0 + e;
    Real d[3][3][4];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int n = 0; n < 4; ++n) d[c][k][n] = 0;
    const Real* fe = F + e * Np * CF + 3 * fld;
#pragma unroll 5
    for (int j = 0; j < Np; ++j) {
      Real a[4], bb[4], cc[4];
      lds4(DrT + j * NpP + 4 * iq, a);
      lds4(DsT + j * NpP + 4 * iq, bb);
      lds4(DtT + j * NpP + 4 * iq, cc);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const Real v = fe[j * CF + c];
#pragma unroll
        for (int n = 0; n < 4; ++n) {
          d[c][0][n] += a[n] * v;
          d[c][1][n] += bb[n] * v;
          d[c][2][n] += cc[n] * v;
        }
      }
    }
    Real l[3][4];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int n = 0; n < 4; ++n) l[c][n] = 0;
    const Real* fl = FL + e * NF * 6 + (fld == 0 ? 3 : 0);
#pragma unroll 4
    for (int fm = 0; fm < NF; ++fm) {
      Real L[4];
      lds4(LIFTT + fm * NpP + 4 * iq, L);
      const Real f0 = fl[fm * 6], f1 = fl[fm * 6 + 1], f2 = fl[fm * 6 + 2];
#pragma unroll
      for (int n = 0; n < 4; ++n) {
        l[0][n] += L[n] * f0; l[1][n] += L[n] * f1; l[2][n] += L[n] * f2;
      }
    }
    const Real* g = met + e * 12;
    const Real rx = g[0], ry = g[1], rz = g[2], sx = g[3], sy = g[4], sz = g[5];
    const Real tx = g[6], ty = g[7], tz_ = g[8];
    const Real ie = P.mat[eg * 3 + 0], im = P.mat[eg * 3 + 1];
    Real out[3][4];
#pragma unroll
    for (int n = 0; n < 4; ++n) {
#define DX(c) (rx * d[c][0][n] + sx * d[c][1][n] + tx * d[c][2][n])
#define DY(c) (ry * d[c][0][n] + sy * d[c][1][n] + ty * d[c][2][n])
#define DZ(c) (rz * d[c][0][n] + sz * d[c][1][n] + tz_ * d[c][2][n])
      const Real c0 = DY(2) - DZ(1) + l[0][n];
      const Real c1 = DZ(0) - DX(2) + l[1][n];
      const Real c2 = DX(1) - DY(0) + l[2][n];
#undef DX
#undef DY
#undef DZ
      if (fld == 0) { out[0][n] = -im * c0; out[1][n] = -im * c1; out[2][n] = -im * c2; }
      else { out[0][n] = c0; out[1][n] = c1; out[2][n] = c2; }
    }
    if (fld == 1) {
      for (int s = 0; s < nsrc_l; ++s) {
        const SrcDev& sd = P.src[srcl[s]];
        if (sd.elem != eg) continue;
        const Real jt = (Real)dipole_current(sd, tst);
#pragma unroll
        for (int n = 0; n < 4; ++n) {
          const int i = 4 * iq + n;
          const Real w = i < Np ? P.src_w[srcl[s] * Np + i] : Real(0);
#pragma unroll
          for (int c = 0; c < 3; ++c) out[c][n] -= jt * (Real)sd.dir[c] * w;
        }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int n = 0; n < 4; ++n) out[c][n] *= ie;
    }
    const int oc = fld == 0 ? 3 : 0;   // rhs_H lands on components 3..5
    if (!PML) {
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int n = 0; n < 4; ++n) {
          const int i = 4 * iq + n;
          if (i < Np) {
            const int64_t gi = ((int64_t)eg * 6 + oc + c) * Np + i;
            const Real rr = rka * resq[gi] + rdt * out[c][n];
            resq[gi] = rr;
            qout[gi] = F[(e * Np + i) * CF + oc + c] + rkb * rr;
          }
        }
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int n = 0; n < 4; ++n) RS[(e * NpP + 4 * iq + n) * 6 + oc + c] = out[c][n];
    }
  }
  if (PML && STORED) {
  __syncthreads();   // RS complete

  // ---- stored-matrix scheme (eqs. 10-13 with kappa = 1, so (M^a)^-1 M_k and
  // M_k^-1 M^{1/kappa} are the identity): per axis u, 4 nodes per task,
  //   rhs_E = r_E - B_u E_u - C_u P^E_u     rhs_P^E = E_u - D_u P^E_u
  //   rhs_H = r_H - B_u H_u - C_u P^H_u     rhs_P^H = H_u - D_u P^H_u
  // with B_u, C_u, D_u = M_k^-1 M_k^{b_u, c_u, d_u} read from global memory
  for (int task = tid; task < ne * 3 * NIQ; task += NT) {
    const int e = task / (3 * NIQ), r = task - e * 3 * NIQ, u = r / NIQ, iq = r - u * NIQ;
    const int eg = eg0 + e;
    const Real* Bm = P.stored + ((int64_t)(ep0 + e) * 9 + u * 3) * Np * NpP + 4 * iq;
    const Real* Cm = Bm + Np * NpP;
    const Real* Dm = Cm + Np * NpP;
    Real aE[4], aH[4], dE[4], dH[4];
#pragma unroll
    for (int n = 0; n < 4; ++n) aE[n] = aH[n] = dE[n] = dH[n] = 0;
    const Real* fe = F + e * Np * 12;
#pragma unroll 5
    for (int j = 0; j < Np; ++j) {
      Real bb[4], cc[4], dd[4];
      ld4(Bm + j * NpP, bb);
      ld4(Cm + j * NpP, cc);
      ld4(Dm + j * NpP, dd);
      const Real Ej = fe[j * 12 + u], Hj = fe[j * 12 + 3 + u];
      const Real PEj = fe[j * 12 + 6 + u], PHj = fe[j * 12 + 9 + u];
#pragma unroll
      for (int n = 0; n < 4; ++n) {
        aE[n] += bb[n] * Ej + cc[n] * PEj;
        aH[n] += bb[n] * Hj + cc[n] * PHj;
        dE[n] += dd[n] * PEj;
        dH[n] += dd[n] * PHj;
      }
    }
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      const int i = 4 * iq + n;
      if (i >= Np) continue;
      const Real* Fi = F + (e * Np + i) * 12;
      const Real rhs[4] = {RS[(e * NpP + i) * 6 + u] - aE[n], RS[(e * NpP + i) * 6 + 3 + u] - aH[n],
                           Fi[u] - dE[n], Fi[3 + u] - dH[n]};
#pragma unroll
      for (int h = 0; h < 2; ++h) {   // E_u, H_u
        const int64_t gi = ((int64_t)eg * 6 + 3 * h + u) * Np + i;
        const Real rr = rka * resq[gi] + rdt * rhs[h];
        resq[gi] = rr;
        qout[gi] = Fi[3 * h + u] + rkb * rr;
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {   // P^E_u, P^H_u
        const int64_t pi = ((int64_t)(eg - P.K0) * 6 + 3 * h + u) * Np + i;
        const Real rr = rka * resp[pi] + rdt * rhs[2 + h];
        resp[pi] = rr;
        pio[pi] = Fi[6 + 3 * h + u] + rkb * rr;
      }
    }
  }
  }  // stored
  if (PML && !STORED) {
  __syncthreads();   // FL is reused as TZ below

  // ---- phase 3: V_q of the 12 fields at 4 quadrature points; eq. 9 pointwise
  Real* TZ = U;    // [T][NqP][12]: b VE + c VPE | b VH + c VPH | k^-1 VE - d VPE | k^-1 VH - d VPH
  const Real ie0 = Real(1) / (Real)P.eps0;
  for (int task = tid; task < ne * NQQ; task += NT) {
    const int e = task / NQQ, qq = task - e * NQQ;
    Real v[12][4];
#pragma unroll
    for (int c = 0; c < 12; ++c)
#pragma unroll
      for (int n = 0; n < 4; ++n) v[c][n] = 0;
    const Real* fe = F + e * Np * 12;
#pragma unroll 5
    for (int j = 0; j < Np; ++j) {
      Real w[4], f[12];
      lds4(VqT + j * NqP + 4 * qq, w);
      lds4(fe + j * 12, f);
      lds4(fe + j * 12 + 4, f + 4);
      lds4(fe + j * 12 + 8, f + 8);
#pragma unroll
      for (int c = 0; c < 12; ++c)
#pragma unroll
        for (int n = 0; n < 4; ++n) v[c][n] += w[n] * f[c];
    }
    const int64_t sb = (int64_t)(ep0 + e) * 3 * NqP + 4 * qq;
    Real sg[3][4], kp[3][4];
    ld4(P.sig + sb, sg[0]);
    ld4(P.sig + sb + NqP, sg[1]);
    ld4(P.sig + sb + 2 * NqP, sg[2]);
    if (KAPPA) {
      ld4(P.kap + sb, kp[0]);
      ld4(P.kap + sb + NqP, kp[1]);
      ld4(P.kap + sb + 2 * NqP, kp[2]);
    }
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      Real* tzo = TZ + (e * NqP + 4 * qq + n) * 12;
      Real o[12];
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const int vv = (u + 1) % 3, ww = (u + 2) % 3;
        const Real ku = KAPPA ? kp[u][n] : Real(1), kv = KAPPA ? kp[vv][n] : Real(1);
        const Real kw = KAPPA ? kp[ww][n] : Real(1);
        const Real su = sg[u][n], sv = sg[vv][n], sw = sg[ww][n];
        // eq. 9
        const Real a = kv * kw / ku;
        const Real bc = (sv * kw + sw * kv - a * su) / ku * ie0;
        const Real cc = sv * sw * ie0 * ie0 - bc * su * ie0;
        const Real dd = su / ku * ie0;
        const Real ki = Real(1) / ku;
        o[u] = bc * v[u][n] + cc * v[6 + u][n];
        o[3 + u] = bc * v[3 + u][n] + cc * v[9 + u][n];
        o[6 + u] = ki * v[u][n] - dd * v[6 + u][n];
        o[9 + u] = ki * v[3 + u][n] - dd * v[9 + u][n];
      }
#pragma unroll
      for (int c = 0; c < 12; c += 4) sts4(tzo + c, o + c);
    }
  }
  __syncthreads();

  // ---- phase 4: P_q back to the nodes, 4 nodes x 4 of the 12 components:
  //   components 0..5 give s (E,H), 6..11 the right-hand side of P^E, P^H
  for (int task = tid; task < ne * 3 * NIQ; task += NT) {
    const int e = task / (3 * NIQ), r = task - e * 3 * NIQ, cg = r / NIQ, iq = r - cg * NIQ;
    const int eg = eg0 + e;
    Real s[4][4];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int n = 0; n < 4; ++n) s[c][n] = 0;
    const Real* tze = TZ + e * NqP * 12 + 4 * cg;
#pragma unroll 5
    for (int q = 0; q < Nq; ++q) {
      Real w[4], t4[4];
      lds4(PqT + q * NpP + 4 * iq, w);
      lds4(tze + q * 12, t4);
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int n = 0; n < 4; ++n) s[c][n] += w[n] * t4[c];
    }
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      const int i = 4 * iq + n;
      if (i >= Np) continue;
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        const int c = 4 * cg + cc;
        if (c < 6) {
          const Real wv = RS[(e * NpP + i) * 6 + c] - s[cc][n];
          if (!KAPPA) {
            const int64_t gi = ((int64_t)eg * 6 + c) * Np + i;
            const Real rr = rka * resq[gi] + rdt * wv;
            resq[gi] = rr;
            qout[gi] = F[(e * Np + i) * 12 + c] + rkb * rr;
          } else {
            RS[(e * NpP + i) * 6 + c] = wv;
          }
        } else {
          const int64_t pi = ((int64_t)(eg - P.K0) * 6 + c - 6) * Np + i;
          const Real rr = rka * resp[pi] + rdt * s[cc][n];
          resp[pi] = rr;
          pio[pi] = F[(e * Np + i) * 12 + c] + rkb * rr;
        }
      }
    }
  }
  if (KAPPA) {
  __syncthreads();

  // ---- phase 5: a^{-1} V_q (Cbar/eps - s) at the quadrature points
  for (int task = tid; task < ne * NQQ; task += NT) {
    const int e = task / NQQ, qq = task - e * NQQ;
    Real v[6][4];
#pragma unroll
    for (int c = 0; c < 6; ++c)
#pragma unroll
      for (int n = 0; n < 4; ++n) v[c][n] = 0;
    const Real* re = RS + e * NpP * 6;
    for (int j = 0; j < Np; ++j) {
      Real w[4], f[6];
      lds4(VqT + j * NqP + 4 * qq, w);
      lds2(re + j * 6, f);
      lds2(re + j * 6 + 2, f + 2);
      lds2(re + j * 6 + 4, f + 4);
#pragma unroll
      for (int c = 0; c < 6; ++c)
#pragma unroll
        for (int n = 0; n < 4; ++n) v[c][n] += w[n] * f[c];
    }
    const int64_t sb = (int64_t)(ep0 + e) * 3 * NqP + 4 * qq;
    Real kp[3][4];
    ld4(P.kap + sb, kp[0]);
    ld4(P.kap + sb + NqP, kp[1]);
    ld4(P.kap + sb + 2 * NqP, kp[2]);
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      Real* tzo = TZ + (e * NqP + 4 * qq + n) * 12;
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const Real ainv = kp[u][n] / (kp[(u + 1) % 3][n] * kp[(u + 2) % 3][n]);
        tzo[u] = ainv * v[u][n];
        tzo[3 + u] = ainv * v[3 + u][n];
      }
    }
  }
  __syncthreads();

  // ---- phase 6: P_q back to the nodes, E/H update
  for (int task = tid; task < ne * NIQ; task += NT) {
    const int e = task / NIQ, iq = task - e * NIQ;
    const int eg = eg0 + e;
    Real s[6][4];
#pragma unroll
    for (int c = 0; c < 6; ++c)
#pragma unroll
      for (int n = 0; n < 4; ++n) s[c][n] = 0;
    const Real* tze = TZ + e * NqP * 12;
    for (int q = 0; q < Nq; ++q) {
      Real w[4], t6[6];
      lds4(PqT + q * NpP + 4 * iq, w);
      lds2(tze + q * 12, t6);
      lds2(tze + q * 12 + 2, t6 + 2);
      lds2(tze + q * 12 + 4, t6 + 4);
#pragma unroll
      for (int c = 0; c < 6; ++c)
#pragma unroll
        for (int n = 0; n < 4; ++n) s[c][n] += w[n] * t6[c];
    }
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      const int i = 4 * iq + n;
      if (i >= Np) continue;
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        const int64_t gi = ((int64_t)eg * 6 + c) * Np + i;
        const Real rr = rka * resq[gi] + rdt * s[c][n];
        resq[gi] = rr;
        qout[gi] = F[(e * Np + i) * 12 + c] + rkb * rr;
      }
    }
  }
  }  // KAPPA
  }  // PML
  }  // tile loop
}

template <typename Real, int N, bool PML, bool KAPPA, bool STORED = false>
__global__ void __launch_bounds__(Tile<Real, N, PML>::THREADS)
stage_kernel(const StageParams<Real> P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  stage_body<Real, N, PML, KAPPA, STORED, 0>(P, smem_raw, blockIdx.x, gridDim.x);
}

template <typename Real, int N, bool PML, bool KAPPA, bool STORED = false>
static cudaError_t configure_one() {
  using TL = Tile<Real, N, PML>;
  return cudaFuncSetAttribute(stage_kernel<Real, N, PML, KAPPA, STORED>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TL::smem);
}

// resident blocks per SM of one stage-kernel instance (cached per instance)
template <typename Real, int N, bool PML, bool KAPPA, bool STORED = false>
static int resident_blocks() {
  static int cached = 0;
  if (cached == 0) {
    using TL = Tile<Real, N, PML>;
    int nb = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, stage_kernel<Real, N, PML, KAPPA, STORED>,
                                                      TL::THREADS, TL::smem) != cudaSuccess ||
        nb < 1)
      nb = 1;
    cached = nb * (sms > 0 ? sms : 1);
  }
  return cached;
}

template <typename Real, int N, bool PML, bool KAPPA, bool STORED = false>
static cudaError_t launch_one(const StageParams<Real>& P, int nb, cudaStream_t s) {
  using TL = Tile<Real, N, PML>;
  if (P.n_elem <= 0) return cudaSuccess;
  StageParams<Real> Q = P;
  Q.nb = nb;
  const long long tiles = (long long)((P.n_elem + TL::T - 1) / TL::T) * nb;
  const int grid =
      (int)std::min<long long>(tiles, resident_blocks<Real, N, PML, KAPPA, STORED>());
  stage_kernel<Real, N, PML, KAPPA, STORED><<<grid, TL::THREADS, TL::smem, s>>>(Q);
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

// ------------------------------------------------------------ grouped launch
// One launch advances every element class of every context of a group by one
// stage (FP32).  Every block starts on the (context, class) item the static
// split gives it, takes that item's tiles from its counter, then moves on to
// the items that still have tiles, restaging the operators once per item.
// Two block shapes: 256 threads (two blocks per SM) or 512 (one).

// dynamic shared memory of one item with `tile` elements per tile
template <int N, bool PML, int NT>
size_t group_smem_one(int tile) {
  using TL = Tile<float, N, PML, NT>;
  const int t = tile > 0 && tile < TL::T ? tile : TL::T;
  return (size_t)(TL::ops_sz + t * TL::per_elem) * sizeof(float) + 64 * sizeof(int);
}

template <int NT>
size_t group_smem_nt(int N, bool pml, int tile) {
  switch (N) {
    case 1: return pml ? group_smem_one<1, true, NT>(tile) : group_smem_one<1, false, NT>(tile);
    case 2: return pml ? group_smem_one<2, true, NT>(tile) : group_smem_one<2, false, NT>(tile);
    case 3: return pml ? group_smem_one<3, true, NT>(tile) : group_smem_one<3, false, NT>(tile);
    case 4: return pml ? group_smem_one<4, true, NT>(tile) : group_smem_one<4, false, NT>(tile);
    case 5: return pml ? group_smem_one<5, true, NT>(tile) : group_smem_one<5, false, NT>(tile);
    default: return 0;
  }
}

size_t group_smem_bytes(int N, bool pml, int tile, int threads) {
  return threads == 512 ? group_smem_nt<512>(N, pml, tile) : group_smem_nt<256>(N, pml, tile);
}

template <int NT>
int group_tile_nt(int N, bool pml) {
  switch (N) {
    case 1: return pml ? Tile<float, 1, true, NT>::T : Tile<float, 1, false, NT>::T;
    case 2: return pml ? Tile<float, 2, true, NT>::T : Tile<float, 2, false, NT>::T;
    case 3: return pml ? Tile<float, 3, true, NT>::T : Tile<float, 3, false, NT>::T;
    case 4: return pml ? Tile<float, 4, true, NT>::T : Tile<float, 4, false, NT>::T;
    case 5: return pml ? Tile<float, 5, true, NT>::T : Tile<float, 5, false, NT>::T;
    default: return 0;
  }
}

int group_tile_max(int N, bool pml, int threads) {
  return threads == 512 ? group_tile_nt<512>(N, pml) : group_tile_nt<256>(N, pml);
}

template <int NT>
__global__ void __launch_bounds__(NT, NT == 256 ? 2 : 1) group_stage_kernel(const GroupParams G) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ StageParams<float> P;
  __shared__ int start;
  __shared__ int go;
  if (threadIdx.x == 0) {
    int it = 0;
    while (it + 1 < G.nitems && (int)blockIdx.x >= G.first[it + 1]) ++it;
    start = it;
  }
  for (int k = 0; k < G.nitems; ++k) {
    __syncthreads();   // start is set; the previous item's body is done with P and go
    const int it = (start + k) % G.nitems;
    // one thread decides whether the item still has tiles, so that the whole
    // block takes the same path through the barriers
    if (threadIdx.x == 0) {
      go = *reinterpret_cast<volatile const int*>(G.counter + it) < G.ntiles[it];
      if (go) P = G.p[it];
    }
    __syncthreads();
    if (!go) continue;
    int* dyn = G.counter + it;
#define WADG_GROUP_CASE(NN)                                                               \
  case NN * 4 + 0: stage_body<float, NN, false, false, false, NT>(P, smem_raw, 0, 1, dyn); break; \
  case NN * 4 + 1: stage_body<float, NN, true, false, false, NT>(P, smem_raw, 0, 1, dyn); break;  \
  case NN * 4 + 2: stage_body<float, NN, true, true, false, NT>(P, smem_raw, 0, 1, dyn); break;
    switch (G.code[it]) {
      WADG_GROUP_CASE(1)
      WADG_GROUP_CASE(2)
      WADG_GROUP_CASE(3)
      WADG_GROUP_CASE(4)
      WADG_GROUP_CASE(5)
      default: break;
    }
#undef WADG_GROUP_CASE
  }
}

cudaError_t configure_group_kernel() {
  size_t m256 = 0, m512 = 0;
  for (int N = 1; N <= 5; ++N)
    for (int pml = 0; pml < 2; ++pml) {
      m256 = std::max(m256, group_smem_bytes(N, pml != 0, 0, 256));
      m512 = std::max(m512, group_smem_bytes(N, pml != 0, 0, 512));
    }
  cudaError_t e = cudaFuncSetAttribute(group_stage_kernel<256>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)m256);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(group_stage_kernel<512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)m512);
}

int group_blocks_per_sm(size_t smem, int threads) {
  int nb = 0;
  cudaError_t e = threads == 512
      ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, group_stage_kernel<512>, 512, smem)
      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, group_stage_kernel<256>, 256, smem);
  if (e != cudaSuccess || nb < 1) nb = 1;
  return nb;
}

cudaError_t launch_group_stage(const GroupParams& G, int nblocks, size_t smem, int threads,
                               cudaStream_t s) {
  if (nblocks <= 0) return cudaSuccess;
  if (threads == 512) group_stage_kernel<512><<<nblocks, 512, smem, s>>>(G);
  else group_stage_kernel<256><<<nblocks, 256, smem, s>>>(G);
  return cudaGetLastError();
}

// ------------------------------------------------------- stored-matrix scheme
template <typename Real>
cudaError_t configure_stored_kernels(int N) {
  switch (N) {
    case 1: return configure_one<Real, 1, true, false, true>();
    case 2: return configure_one<Real, 2, true, false, true>();
    case 3: return configure_one<Real, 3, true, false, true>();
    case 4: return configure_one<Real, 4, true, false, true>();
    case 5: return configure_one<Real, 5, true, false, true>();
    default: return cudaErrorInvalidValue;
  }
}
template cudaError_t configure_stored_kernels<double>(int);
template cudaError_t configure_stored_kernels<float>(int);

template <typename Real>
cudaError_t launch_stage_stored(int N, const StageParams<Real>& P, int nb, cudaStream_t s) {
  switch (N) {
    case 1: return launch_one<Real, 1, true, false, true>(P, nb, s);
    case 2: return launch_one<Real, 2, true, false, true>(P, nb, s);
    case 3: return launch_one<Real, 3, true, false, true>(P, nb, s);
    case 4: return launch_one<Real, 4, true, false, true>(P, nb, s);
    case 5: return launch_one<Real, 5, true, false, true>(P, nb, s);
    default: return cudaErrorInvalidValue;
  }
}
template cudaError_t launch_stage_stored<double>(int, const StageParams<double>&, int, cudaStream_t);
template cudaError_t launch_stage_stored<float>(int, const StageParams<float>&, int, cudaStream_t);

// Stored operators M_k^-1 M_k^{alpha} = P_h diag(alpha(x_h)) V_h for alpha in
// {b_u, c_u, d_u} of eq. 9 (kappa = 1), u = x, y, z, of TE elements per block,
// in double precision.  The rule's points are processed in chunks staged in
// shared memory (P_h and V_h columns, the nine coefficient samples of each
// element); every thread accumulates ENT entries (i, j) of the nine operators
// of each of its block's elements in registers.
template <int N>
struct StoredSetup {
  static constexpr int Np = (N + 1) * (N + 2) * (N + 3) / 6;
  static constexpr int NpP = (Np + 3) & ~3;
  static constexpr int THREADS = 256;
  static constexpr int ENT = (Np * Np + THREADS - 1) / THREADS;
  static constexpr int TE = ENT <= 2 ? 4 : (ENT <= 5 ? 2 : 1);
  static constexpr int HC = 32;
};

template <typename Real, int N>
__global__ void __launch_bounds__(StoredSetup<N>::THREADS)
stored_ops_kernel(int K1, int K0, int Nh, const double* verts, const double* prof,
                  const double* rh, const double* Ph, const double* Vh, Real* out) {
  using S = StoredSetup<N>;
  constexpr int Np = S::Np, NpP = S::NpP, NT = S::THREADS, ENT = S::ENT, TE = S::TE, HC = S::HC;
  __shared__ double PhC[Np][HC];
  __shared__ double VhC[HC][Np];
  __shared__ double al[TE][9][HC];   // [element][3 u + kind][point]: b_u, c_u, d_u
  const int tid = threadIdx.x;
  const int e0 = blockIdx.x * TE;
  double acc[TE][9][ENT];
#pragma unroll
  for (int t = 0; t < TE; ++t)
#pragma unroll
    for (int m = 0; m < 9; ++m)
#pragma unroll
      for (int k = 0; k < ENT; ++k) acc[t][m][k] = 0.0;
  const double ie0 = 1.0 / prof[15];
  for (int h0 = 0; h0 < Nh; h0 += HC) {
    __syncthreads();   // previous chunk consumed
    for (int idx = tid; idx < Np * HC; idx += NT) {
      const int i = idx / HC, hh = idx - i * HC;
      PhC[i][hh] = h0 + hh < Nh ? Ph[(int64_t)i * Nh + h0 + hh] : 0.0;
    }
    for (int idx = tid; idx < HC * Np; idx += NT) {
      const int hh = idx / Np, j = idx - hh * Np;
      VhC[hh][j] = h0 + hh < Nh ? Vh[(int64_t)(h0 + hh) * Np + j] : 0.0;
    }
    for (int idx = tid; idx < TE * HC; idx += NT) {
      const int t = idx / HC, hh = idx - t * HC;
      double sg[3] = {0.0, 0.0, 0.0};
      if (e0 + t < K1 && h0 + hh < Nh) {
        const double* v = verts + (int64_t)(K0 + e0 + t) * 12;
        const double r = rh[(h0 + hh) * 3], s_ = rh[(h0 + hh) * 3 + 1], tt = rh[(h0 + hh) * 3 + 2];
        const double l0 = -0.5 * (1 + r + s_ + tt), l1 = 0.5 * (1 + r), l2 = 0.5 * (1 + s_),
                     l3 = 0.5 * (1 + tt);
        for (int u = 0; u < 3; ++u) {
          const double x = l0 * v[u] + l1 * v[3 + u] + l2 * v[6 + u] + l3 * v[9 + u];
          const double d = (fabs(x) - prof[u]) / prof[3 + u];
          sg[u] = d > 0 ? prof[6 + u] * pow(d, prof[9 + u]) : 0.0;
        }
      }
      for (int u = 0; u < 3; ++u) {
        const double su = sg[u], sv = sg[(u + 1) % 3], sw = sg[(u + 2) % 3];
        const double b = (sv + sw - su) * ie0;              // eq. 9, kappa = 1
        al[t][3 * u][hh] = b;
        al[t][3 * u + 1][hh] = sv * sw * ie0 * ie0 - b * su * ie0;
        al[t][3 * u + 2][hh] = su * ie0;
      }
    }
    __syncthreads();
    for (int hh = 0; hh < HC; ++hh) {
#pragma unroll
      for (int k = 0; k < ENT; ++k) {
        const int ent = tid + k * NT;
        if (ent >= Np * Np) continue;
        const int i = ent / Np, j = ent - i * Np;
        const double w = PhC[i][hh] * VhC[hh][j];
#pragma unroll
        for (int t = 0; t < TE; ++t)
#pragma unroll
          for (int m = 0; m < 9; ++m) acc[t][m][k] += w * al[t][m][hh];
      }
    }
  }
#pragma unroll
  for (int t = 0; t < TE; ++t) {
    if (e0 + t >= K1) continue;
#pragma unroll
    for (int k = 0; k < ENT; ++k) {
      const int ent = tid + k * NT;
      if (ent >= Np * Np) continue;
      const int i = ent / Np, j = ent - i * Np;
#pragma unroll
      for (int m = 0; m < 9; ++m)   // transposed: row j of the stored block is column j
        out[(((int64_t)(e0 + t) * 9 + m) * Np + j) * NpP + i] = (Real)acc[t][m][k];
    }
  }
}

template <typename Real>
cudaError_t launch_stored_ops(int N, int K1, int K0, const double* verts, const double* prof,
                              const double* rh, const double* Ph, const double* Vh, int Nh,
                              Real* out, cudaStream_t s) {
  if (K1 <= 0) return cudaSuccess;
#define WADG_STORED_CASE(NN)                                                              \
  case NN: {                                                                              \
    using S = StoredSetup<NN>;                                                            \
    stored_ops_kernel<Real, NN><<<(K1 + S::TE - 1) / S::TE, S::THREADS, 0, s>>>(          \
        K1, K0, Nh, verts, prof, rh, Ph, Vh, out);                                        \
    return cudaGetLastError();                                                            \
  }
  switch (N) {
    WADG_STORED_CASE(1)
    WADG_STORED_CASE(2)
    WADG_STORED_CASE(3)
    WADG_STORED_CASE(4)
    WADG_STORED_CASE(5)
    default: return cudaErrorInvalidValue;
  }
#undef WADG_STORED_CASE
}
template cudaError_t launch_stored_ops<double>(int, int, int, const double*, const double*,
                                               const double*, const double*, const double*, int,
                                               double*, cudaStream_t);
template cudaError_t launch_stored_ops<float>(int, int, int, const double*, const double*,
                                              const double*, const double*, const double*, int,
                                              float*, cudaStream_t);

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
__global__ void pml_samples_kernel(int Nq, int NqP, int K1, int K0, const double* verts,
                                   const double* rq, const double* prof, Real* sig,
                                   Real* kap, bool element_constant) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)K1 * NqP) return;
  const int e = (int)(idx / NqP), q = (int)(idx - (int64_t)e * NqP);
  if (q >= Nq) {   // padding of the quadrature axis
    for (int u = 0; u < 3; ++u) {
      sig[((int64_t)e * 3 + u) * NqP + q] = Real(0);
      if (kap) kap[((int64_t)e * 3 + u) * NqP + q] = Real(1);
    }
    return;
  }
  const double* v = verts + (int64_t)(K0 + e) * 12;
  // the quadrature node, or the centroid for element-constant coefficients
  const double r = element_constant ? -0.5 : rq[q * 3];
  const double s = element_constant ? -0.5 : rq[q * 3 + 1];
  const double t = element_constant ? -0.5 : rq[q * 3 + 2];
  const double l0 = -0.5 * (1 + r + s + t), l1 = 0.5 * (1 + r), l2 = 0.5 * (1 + s),
               l3 = 0.5 * (1 + t);
  for (int u = 0; u < 3; ++u) {
    const double x = l0 * v[u] + l1 * v[3 + u] + l2 * v[6 + u] + l3 * v[9 + u];
    const double d = (fabs(x) - prof[u]) / prof[3 + u];
    double g = 0.0;
    if (d > 0) g = pow(d, prof[9 + u]);
    sig[((int64_t)e * 3 + u) * NqP + q] = (Real)(prof[6 + u] * g);
    if (kap) kap[((int64_t)e * 3 + u) * NqP + q] = (Real)(1.0 + (prof[12 + u] - 1.0) * g);
  }
}

template <typename Real>
cudaError_t launch_pml_samples(int Nq, int K1, int K0, const double* verts, const double* rq,
                               const double* prof, Real* sig, Real* kap, bool element_constant,
                               cudaStream_t s) {
  const int NqP = (Nq + 3) & ~3;
  const int64_t n = (int64_t)K1 * NqP;
  if (n == 0) return cudaSuccess;
  const int th = 256;
  pml_samples_kernel<Real><<<(unsigned)((n + th - 1) / th), th, 0, s>>>(Nq, NqP, K1, K0, verts,
                                                                       rq, prof, sig, kap,
                                                                       element_constant);
  return cudaGetLastError();
}
template cudaError_t launch_pml_samples<double>(int, int, int, const double*, const double*,
                                                const double*, double*, double*, bool,
                                                cudaStream_t);
template cudaError_t launch_pml_samples<float>(int, int, int, const double*, const double*,
                                               const double*, float*, float*, bool, cudaStream_t);

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
