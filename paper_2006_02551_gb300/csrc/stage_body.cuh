// Body of the CUDA-core DGTD stage (shared by the per-class launches in
// kernels.cu and the grouped launch in group.cu): one pass over a tile of
// elements computes the right-hand side of the semi-discrete system and
// applies the low-storage Runge-Kutta update.
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
#pragma once
#include "kernels.cuh"

#include <algorithm>
#include <cstdio>
#include <type_traits>

namespace wadg {

template <int N, int QC = 0>
struct Dims {
  static constexpr int Np = (N + 1) * (N + 2) * (N + 3) / 6;
  static constexpr int Nfp = (N + 1) * (N + 2) / 2;
  static constexpr int Nq = quad_capacity(N, QC);   // volume quadrature points
  static constexpr int NF = 4 * Nfp;
  static constexpr int NpP = (Np + 3) & ~3;   // padded to whole quads
  static constexpr int NqP = (Nq + 3) & ~3;
  static constexpr int NIQ = NpP / 4;         // node quads
  static constexpr int NQQ = NqP / 4;         // quadrature-point quads
};

// Launch configuration: persistent blocks, the reference operators staged in
// shared memory once per block, tiles of T elements processed in a loop.
template <typename Real, int N, bool PML, int NT_ = 0, int QC = 0>
struct Tile {
  using D = Dims<N, QC>;
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
template <typename Real, int N, bool PML, bool KAPPA, bool STORED, int NT_, int QC = 0>
__device__ __forceinline__ void stage_body(const StageParams<Real>& P, unsigned char* smem_raw,
                                           int bid, int nblk, int* dyn = nullptr) {
  using D = Dims<N, QC>;
  constexpr int Np = D::Np, Nfp = D::Nfp, Nq = D::Nq, NF = D::NF;
  constexpr int NpP = D::NpP, NqP = D::NqP, NIQ = D::NIQ, NQQ = D::NQQ;
  using TL = Tile<Real, N, PML, NT_, QC>;
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

  // dynamic schedule: thread 0 claims the next tile at the start of the
  // current one and publishes it at the end, so the atomic's round trip
  // overlaps the tile's work (a claim past the last tile is left unused)
  __shared__ int dyn_tile;
  int claimed = 0;
  auto claim = [&]() {
    if (dyn && tid == 0) claimed = atomicAdd(dyn, 1);
  };
  auto next_tile = [&](int cur) -> int {
    if (!dyn) return cur < 0 ? bid : cur + nblk;
    __syncthreads();   // every thread has read the previous value
    if (tid == 0) dyn_tile = claimed;
    __syncthreads();
    return dyn_tile;
  };
  claim();
  for (int tile = next_tile(-1); tile < ntiles; tile = next_tile(tile)) {
  claim();
  const int b = tile / tiles_per_batch;
  const int t0 = (tile - b * tiles_per_batch) * TE;
  const int ne = min(TE, P.n_elem - t0);
  const int eg0 = P.e_begin + t0;
  const int ep0 = eg0 - P.K0;
  const Real* qin = P.qin + (int64_t)b * P.strideQ;
  Real* qout = P.qout + (int64_t)b * P.strideQ;
  Real* resq = P.resq + (int64_t)b * P.strideQ;
  Real* pio = P.p + (int64_t)b * P.strideP;
  Real* pout = (P.pout ? P.pout : P.p) + (int64_t)b * P.strideP;   // read in phase 0, written last
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
    const int code = nb >= 0 ? P.code[eg * 4 + f] : 0;
    const bool face_ok =
        nb >= 0 && WADG_INDEX_OK(nb < P.strideQ / (6 * Np) && code < 24, P.err);
    const int np2 = face_ok ? fperm[(f * 24 + code) * Nfp + m] : 0;
    if (face_ok && WADG_INDEX_OK(np2 < Np, P.err)) {
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

  // ---- stored-matrix scheme (eqs. 10-13): per axis u, 4 nodes per task,
  //   r_E = Cbar(H)/eps - B_u E_u - C_u P^E_u     rhs_P^E = K_u E_u - D_u P^E_u
  //   r_H = -Cbar(E)/mu - B_u H_u - C_u P^H_u     rhs_P^H = K_u H_u - D_u P^H_u
  //   rhs_E = A_u^-1 r_E,  rhs_H = A_u^-1 r_H
  // with B_u, C_u, D_u = M_k^-1 M_k^{b_u, c_u, d_u}, K_u = M_k^-1 M_k^{1/kappa_u}
  // and A_u^-1 = (M_k^{a_u})^-1 M_k read from global memory; with kappa = 1,
  // K_u and A_u^-1 are the identity and are not stored
  constexpr int NBK = KAPPA ? 5 : 3;
  for (int task = tid; task < ne * 3 * NIQ; task += NT) {
    const int e = task / (3 * NIQ), r = task - e * 3 * NIQ, u = r / NIQ, iq = r - u * NIQ;
    const int eg = eg0 + e;
    const Real* Bm = P.stored + ((int64_t)(ep0 + e) * 3 + u) * NBK * Np * NpP + 4 * iq;
    const Real* Cm = Bm + Np * NpP;
    const Real* Dm = Cm + Np * NpP;
    const Real* Km = Dm + Np * NpP;   // kappa != 1 only
    Real aE[4], aH[4], dE[4], dH[4], kE[4], kH[4];
#pragma unroll
    for (int n = 0; n < 4; ++n) aE[n] = aH[n] = dE[n] = dH[n] = kE[n] = kH[n] = 0;
    const Real* fe = F + e * Np * 12;
#pragma unroll 5
    for (int j = 0; j < Np; ++j) {
      Real bb[4], cc[4], dd[4], kk[4];
      ld4(Bm + j * NpP, bb);
      ld4(Cm + j * NpP, cc);
      ld4(Dm + j * NpP, dd);
      if (KAPPA) ld4(Km + j * NpP, kk);
      const Real Ej = fe[j * 12 + u], Hj = fe[j * 12 + 3 + u];
      const Real PEj = fe[j * 12 + 6 + u], PHj = fe[j * 12 + 9 + u];
#pragma unroll
      for (int n = 0; n < 4; ++n) {
        aE[n] += bb[n] * Ej + cc[n] * PEj;
        aH[n] += bb[n] * Hj + cc[n] * PHj;
        dE[n] += dd[n] * PEj;
        dH[n] += dd[n] * PHj;
        if (KAPPA) {
          kE[n] += kk[n] * Ej;
          kH[n] += kk[n] * Hj;
        }
      }
    }
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      const int i = 4 * iq + n;
      if (i >= Np) continue;
      const Real* Fi = F + (e * Np + i) * 12;
      const Real rhs[4] = {RS[(e * NpP + i) * 6 + u] - aE[n], RS[(e * NpP + i) * 6 + 3 + u] - aH[n],
                           (KAPPA ? kE[n] : Fi[u]) - dE[n], (KAPPA ? kH[n] : Fi[3 + u]) - dH[n]};
      if (KAPPA) {   // r_E, r_H of node i, for A_u^-1 below
        RS[(e * NpP + i) * 6 + u] = rhs[0];
        RS[(e * NpP + i) * 6 + 3 + u] = rhs[1];
      } else {
#pragma unroll
        for (int h = 0; h < 2; ++h) {   // E_u, H_u
          const int64_t gi = ((int64_t)eg * 6 + 3 * h + u) * Np + i;
          const Real rr = rka * resq[gi] + rdt * rhs[h];
          resq[gi] = rr;
          qout[gi] = Fi[3 * h + u] + rkb * rr;
        }
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {   // P^E_u, P^H_u
        const int64_t pi = ((int64_t)(eg - P.K0) * 6 + 3 * h + u) * Np + i;
        const Real rr = rka * resp[pi] + rdt * rhs[2 + h];
        resp[pi] = rr;
        pout[pi] = Fi[6 + 3 * h + u] + rkb * rr;
      }
    }
  }
  if (KAPPA) {
  __syncthreads();   // every r_E, r_H of the tile is in RS
  for (int task = tid; task < ne * 3 * NIQ; task += NT) {
    const int e = task / (3 * NIQ), r = task - e * 3 * NIQ, u = r / NIQ, iq = r - u * NIQ;
    const int eg = eg0 + e;
    const Real* Am = P.stored + (((int64_t)(ep0 + e) * 3 + u) * NBK + 4) * Np * NpP + 4 * iq;
    Real sE[4] = {0, 0, 0, 0}, sH[4] = {0, 0, 0, 0};
#pragma unroll 5
    for (int j = 0; j < Np; ++j) {
      Real aa[4];
      ld4(Am + j * NpP, aa);
      const Real rEj = RS[(e * NpP + j) * 6 + u], rHj = RS[(e * NpP + j) * 6 + 3 + u];
#pragma unroll
      for (int n = 0; n < 4; ++n) {
        sE[n] += aa[n] * rEj;
        sH[n] += aa[n] * rHj;
      }
    }
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      const int i = 4 * iq + n;
      if (i >= Np) continue;
      const Real* Fi = F + (e * Np + i) * 12;
      const Real rhs[2] = {sE[n], sH[n]};
#pragma unroll
      for (int h = 0; h < 2; ++h) {   // E_u, H_u
        const int64_t gi = ((int64_t)eg * 6 + 3 * h + u) * Np + i;
        const Real rr = rka * resq[gi] + rdt * rhs[h];
        resq[gi] = rr;
        qout[gi] = Fi[3 * h + u] + rkb * rr;
      }
    }
  }
  }  // KAPPA
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
          pout[pi] = F[(e * Np + i) * 12 + c] + rkb * rr;
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

}  // namespace wadg
