// Tensor-core stage kernels with row-owned epilogues (sm_103a: tcgen05 with
// TF32 or BF16 operands, FP32 accumulation in tensor memory, FP32 state),
// for contexts with a compact volume rule (quad_capacity class 1).
//
// Every contraction of the stage is one product
//     D[row][n] = sum_k A[row][k] * B[n][k]
// whose A operand is the tile's field data, one row per (element,
// component), and whose B operand is the reference operator (row n = output
// node, quadrature point or stacked derivative).  A tile is T = 16 elements
// (8 at N = 5) of 8 rows each (Ex, Ey, Ez, Hx, Hy, Hz and two zero rows), so
// the M = 128 rows of a product are the 128 tensor-memory lanes and the
// thread that owns lane (e, c) receives every output of every product for
// its element and component:
//   F rows (E, H)   x [Dr; Ds; Dt]  -> reference derivatives   (eqs. 16, 17)
//   flux rows       x LIFT          -> surface term
//   F rows          x V_q           -> E, H at the quadrature points (eqs. 26-29)
//   P rows (P^E, P^H) x V_q         -> P at the quadrature points
//   T rows (t)      x P_q           -> s, the weight-adjusted term of E, H
//   Z rows (z)      x P_q           -> right-hand side of P
// Lane (e, c) owns E/H component c and P component c of element e, so
// eq. 9 at the quadrature points is local to the thread; the curl needs the
// other components' derivatives, which the six lanes of an element exchange
// by warp shuffles.  No product output goes through shared memory and the
// epilogue warps never synchronise with each other: one issuing thread
// chains the products on mbarriers.
//
// Warp roles: epilogue warps (two per tensor-memory lane quadrant that holds
// live rows, splitting the nodes and quadrature points of their rows in
// halves), flux warps (upwind flux into the LIFT operand) and one issuing
// warp whose first lane stages each tile with bulk copies (and prefetches
// the next tile into L2), issues every product and writes the results back
// with bulk copies.  Every wait is bounded; on timeout the kernel records an
// error, drains its copies and products and releases its tensor memory.
#include "kernels.cuh"
#include "tc_ptx.cuh"

#include <algorithm>
#include <cstdint>

namespace wadg {
namespace tc {

constexpr int rup4(int x) { return (x + 3) & ~3; }

template <int N, bool PML, bool BF>
struct RPlan {
  using O = OpT<BF>;
  static constexpr int Np = (N + 1) * (N + 2) * (N + 3) / 6;
  static constexpr int Nfp = (N + 1) * (N + 2) / 2;
  static constexpr int NF = 4 * Nfp;
  static constexpr int Nq = compact_nq(N);          // capacity of the compact class
  static constexpr int NqP = (Nq + 3) & ~3;         // stride of the sigma samples
  static constexpr int CW = O::CW, KS = O::KS;
  __host__ __device__ static constexpr int rupK(int x) { return (x + KS - 1) / KS * KS; }
  static constexpr int NpK = rupK(Np), NFK = rupK(NF), NqK = rupK(Nq);
  static constexpr int T = N <= 4 ? 16 : 8;         // elements per tile
  static constexpr int LIVE = 8 * T;                // live rows / lanes
  static constexpr int NpA = rup4(Np);              // stacked derivative block
  // product widths (columns): V_q, stacked derivatives, LIFT, P_q
  static constexpr int NV = rup16(Nq), ND = rup16(3 * NpA), NL = rup16(Np), NPQ = rup16(Np);
  static_assert(NPQ <= NV, "P_q outputs reuse the V_q columns");
  static_assert(NV <= 256 && ND <= 256, "product width");
  // tensor-memory columns
  static constexpr uint32_t cVF = 0, cVP = PML ? NV : 0;
  static constexpr uint32_t cD = PML ? 2 * NV : 0, cL = cD + ND;
  static constexpr uint32_t COLS = cL + NL;
  static constexpr uint32_t TMEM_COLS =
      COLS <= 32 ? 32 : COLS <= 64 ? 64 : COLS <= 128 ? 128 : COLS <= 256 ? 256 : 512;
  static_assert(COLS <= 512, "tensor-memory columns");
  // canonical K-major layout without swizzle: 8-row x 16-byte core matrices,
  // K-adjacent core matrices 128 bytes apart, 8-row groups SB(K) apart
  __host__ __device__ static constexpr uint32_t SB(int K) { return (uint32_t)(K / CW) * 128u; }
  static constexpr uint32_t SBF = SB(NpK), SBT = SB(NqK), SBL = SB(NFK);
  // B operands (the reference operators, staged once per block)
  static constexpr uint32_t oBD = 0;
  static constexpr uint32_t oBL = oBD + (ND / 8) * SBF;
  static constexpr uint32_t oBV = oBL + (NL / 8) * SBL;
  static constexpr uint32_t oBP = oBV + (PML ? (NV / 8) * SBF : 0);
  static constexpr uint32_t oAF = oBP + (PML ? (NPQ / 8) * SBT : 0);
  // A operands: LIVE rows each; an instruction reads 128 rows from its start,
  // the rows past LIVE fall on the buffers that follow (their lanes are
  // never read)
  static constexpr uint32_t AFB = (LIVE / 8) * (PML && SBT > SBF ? SBT : SBF);   // F, then T
  static constexpr uint32_t oAP = oAF + AFB;                                     // P, then Z
  static constexpr uint32_t oAL = oAP + (PML ? AFB : 0);                         // flux
  static constexpr uint32_t oST = oAL + (LIVE / 8) * SBL;
  // staging: each block copied as the 16-byte-aligned cover of its data
  static constexpr uint32_t FB = ((T * 6 * Np * 4 + 15) & ~15) + 16;
  static constexpr uint32_t SGB = PML ? ((T * 3 * NqP * 4 + 15) & ~15) + 16 : 0;
  static constexpr uint32_t GFN = ((T * 64 + 15) & ~15) + 16;
  static constexpr uint32_t GMET = ((T * 72 + 15) & ~15) + 16;
  static constexpr uint32_t GMAT = ((T * 12 + 15) & ~15) + 16;
  static constexpr uint32_t oSQ = oST, oSR = oSQ + FB;
  static constexpr uint32_t oSP = oSR + FB, oSRP = oSP + (PML ? FB : 0);
  static constexpr uint32_t oSSG = oSRP + (PML ? FB : 0);
  static constexpr uint32_t oSFN = oSSG + SGB, oSMET = oSFN + GFN, oSMAT = oSMET + GMET;
  static constexpr uint32_t oMisc = (oSMAT + GMAT + 127) & ~127u;
  // misc: 16 mbarriers | TMEM slot | cached sources (64 x (batch, element)) |
  // face tables (Fmask [NF], fperm [4][24][Nfp])
  static constexpr uint32_t oTabs = 128 + 16 + 512;
  static constexpr uint32_t bytes = oMisc + oTabs + ((100 * Nfp + 15) & ~15u);
  static_assert(oAF + 16 * SBF <= bytes && oAP + 16 * SBF <= bytes, "F / P operand span");
  static_assert(!PML || (oAF + 16 * SBT <= bytes && oAP + 16 * SBT <= bytes), "T / Z span");
  static_assert(oAL + 16 * SBL <= bytes, "flux operand span");
  static_assert(bytes <= 227 * 1024, "shared memory");
  // epilogue warps: two per quadrant of live lanes; flux warps: the rest of 12
  static constexpr int QUADS = LIVE / 32;
  static constexpr int NEW = 2 * QUADS;
  static constexpr int NFW = 12 - NEW;
  static constexpr int THREADS = 32 * 13;
  // node and quadrature-point halves of an epilogue warp (multiples of 4)
  static constexpr int NH = rup4((Np + 1) / 2);
  static constexpr int QH = ((NqK / CW + 1) / 2) * CW;
  static_assert(QH % 4 == 0, "quadrature half");
};

// the epilogue warps' roles: warp w owns lane quadrant w & 3 and half w >> 2
// (T = 16); with T = 8 only quadrants 0 and 1 hold live rows, so the
// epilogue warps are 0, 1, 4, 5 and the others do flux work
template <int QUADS>
__device__ __forceinline__ bool is_epilogue_warp(int w) {
  return w < 8 && (w & 3) < QUADS;
}

template <int N, bool PML, bool BF>
__global__ void __launch_bounds__(RPlan<N, PML, BF>::THREADS, 1)
    tc_rows_kernel(const StageParams<float> P) {
  using PL = RPlan<N, PML, BF>;
  constexpr int Np = PL::Np, Nfp = PL::Nfp, NF = PL::NF, Nq = PL::Nq, T = PL::T;
  constexpr int NpK = PL::NpK, NFK = PL::NFK, NqK = PL::NqK, CW = PL::CW, KS = PL::KS;
  constexpr int NpA = PL::NpA, NqP = PL::NqP;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t sbase = saddr(smem);
  // mbarriers: [0] staging landed, [1] F/P operands ready, [2] flux ready,
  // [3] V_q + derivative products done, [4] LIFT done, [5] T/Z ready,
  // [6] P_q done, [7] results staged, [8] final drain
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + PL::oMisc);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + PL::oMisc + 128);
  int* srcc = reinterpret_cast<int*>(smem + PL::oMisc + 144);   // [64][2]
  unsigned char* tabs = smem + PL::oMisc + PL::oTabs;
  const unsigned char* Fmask = tabs;
  const unsigned char* fperm = tabs + NF;
  constexpr int kSrcCache = 64;

  // ---- prologue: zero operands, stage the operators (B), tables, barriers
  for (uint32_t i = tid; i < PL::oST / 16; i += PL::THREADS)
    reinterpret_cast<float4*>(smem)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();
  {
    // tcops: Dr | Ds | Dt [Np][Np], LIFT [Np][NF], Vq [Nq][Np], Pq [Np][Nq]
    const float* tops = reinterpret_cast<const float*>(P.tcops);
    const float* gL = tops + 3 * Np * Np;
    const float* gVq = gL + Np * NF;
    const float* gPq = gVq + Nq * Np;
    for (int idx = tid; idx < 3 * Np * Np; idx += PL::THREADS) {
      const int d = idx / (Np * Np), r = idx - d * Np * Np, i = r / Np, j = r - i * Np;
      put_op<BF>(smem + PL::oBD + cofs<BF>(d * NpA + i, j, PL::SBF, 128), tops[idx]);
    }
    for (int idx = tid; idx < Np * NF; idx += PL::THREADS) {
      const int i = idx / NF, f = idx - i * NF;
      put_op<BF>(smem + PL::oBL + cofs<BF>(i, f, PL::SBL, 128), gL[idx]);
    }
    if constexpr (PML) {
      for (int idx = tid; idx < Nq * Np; idx += PL::THREADS) {
        const int q = idx / Np, j = idx - q * Np;
        put_op<BF>(smem + PL::oBV + cofs<BF>(q, j, PL::SBF, 128), gVq[idx]);
      }
      for (int idx = tid; idx < Np * Nq; idx += PL::THREADS) {
        const int i = idx / Nq, q = idx - i * Nq;
        put_op<BF>(smem + PL::oBP + cofs<BF>(i, q, PL::SBT, 128), gPq[idx]);
      }
    }
  }
  for (int s = tid; s < min(P.nsrc, kSrcCache); s += PL::THREADS) {
    srcc[2 * s] = P.src[s].batch;
    srcc[2 * s + 1] = P.src[s].elem;
  }
  for (int i = tid; i < 100 * Nfp; i += PL::THREADS) tabs[i] = P.tabs[i];
  if (tid == 0) {
    const uint32_t cnt[9] = {1, (uint32_t)PL::NEW, (uint32_t)PL::NFW, 1, 1, (uint32_t)PL::NEW,
                             1, (uint32_t)PL::NEW, 1};
    for (int i = 0; i < 9; ++i) mbar_init(saddr(mbar + i), cnt[i]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(saddr(tmem_slot), PL::TMEM_COLS);
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  const double tbase = P.t_dev ? *P.t_dev : P.t;
  const double tst = tbase + P.rk_c * P.dt;
  const float rka = (float)P.rk_a, rkb = (float)P.rk_b, rdt = (float)P.dt;
  const int tiles_per_batch = (P.n_elem + T - 1) / T;
  const int ntiles = tiles_per_batch * P.nb;
  bool failed = false;

  // the global blocks of a tile: (address, bytes, staging offset)
  auto tile_geom = [&](int tile, int& b, int& t0, int& ne) {
    b = tile / tiles_per_batch;
    t0 = (tile - b * tiles_per_batch) * T;
    ne = min(T, P.n_elem - t0);
  };
  constexpr int NBLK = PML ? 8 : 5;
  auto tile_blocks = [&](int tile, const unsigned char* (&src)[8], uint32_t (&len)[8],
                         uint32_t (&dst)[8]) {
    int b, t0, ne;
    tile_geom(tile, b, t0, ne);
    const int64_t eg0 = P.e_begin + t0;
    const int64_t oq = (int64_t)b * P.strideQ + eg0 * 6 * Np;
    const int64_t op = (int64_t)b * P.strideP + (eg0 - P.K0) * 6 * Np;
    int a = 0;
    auto add = [&](const void* g, uint32_t n, uint32_t o) {
      src[a] = static_cast<const unsigned char*>(g);
      len[a] = n;
      dst[a] = o;
      ++a;
    };
    add(P.qin + oq, ne * 6 * Np * 4, PL::oSQ);
    add(P.resq + oq, ne * 6 * Np * 4, PL::oSR);
    if constexpr (PML) {
      add(P.p + op, ne * 6 * Np * 4, PL::oSP);
      add(P.resp + op, ne * 6 * Np * 4, PL::oSRP);
      add(P.sig + (eg0 - P.K0) * 3 * NqP, ne * 3 * NqP * 4, PL::oSSG);
    }
    add(P.fnrm + eg0 * 16, ne * 64, PL::oSFN);
    add(P.geo + eg0 * 9, ne * 72, PL::oSMET);
    add(P.mat + eg0 * 3, ne * 12, PL::oSMAT);
  };
  // where the first value of a staged block lands (its cover starts at the
  // 16-byte boundary below it)
  auto staged = [&](uint32_t o, const void* g) {
    return smem + o + (reinterpret_cast<uintptr_t>(g) & 15);
  };

  const int nqd = PL::QUADS;
  if (warp == 12) {
    // ================================================= issuing warp (lane 0)
    if (lane == 0) {
      constexpr uint32_t idV = BF ? idesc_bf16(128, PL::NV) : idesc_tf32(128, PL::NV);
      constexpr uint32_t idD = BF ? idesc_bf16(128, PL::ND) : idesc_tf32(128, PL::ND);
      constexpr uint32_t idL = BF ? idesc_bf16(128, PL::NL) : idesc_tf32(128, PL::NL);
      constexpr uint32_t idP = BF ? idesc_bf16(128, PL::NPQ) : idesc_tf32(128, PL::NPQ);
      auto mma = [](uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
        if constexpr (BF) mma_bf16(d, a, b, id, acc);
        else mma_tf32(d, a, b, id, acc);
      };
      // D[c0..] = A (rows at aoff, K-stride sba) x B (rows at boff, stride sbb), K steps
      auto product = [&](uint32_t col, uint32_t aoff, uint32_t sba, uint32_t boff, uint32_t sbb,
                         int K, uint32_t id) {
        for (int k = 0; k < K / KS; ++k)
          mma(tmem + col, make_desc(sbase + aoff + 256 * k, 128, sba),
              make_desc(sbase + boff + 256 * k, 128, sbb), id, k > 0);
      };
      auto stage_in = [&](int tile) {
        const unsigned char* src[8];
        uint32_t len[8], dst[8];
        tile_blocks(tile, src, len, dst);
        uint32_t lo[8], cl[8], total = 0;
        for (int a = 0; a < NBLK; ++a) {
          lo[a] = (uint32_t)(reinterpret_cast<uintptr_t>(src[a]) & 15);
          cl[a] = (lo[a] + len[a] + 15) & ~15u;
          total += cl[a];
        }
        const uint32_t bar = saddr(mbar + 0);
        fence_async_smem();
        mbar_expect_tx(bar, total);
        for (int a = 0; a < NBLK; ++a) bulk_g2s(sbase + dst[a], src[a] - lo[a], cl[a], bar);
      };
      auto prefetch = [&](int tile) {
        const unsigned char* src[8];
        uint32_t len[8], dst[8];
        tile_blocks(tile, src, len, dst);
        for (int a = 0; a < NBLK; ++a) {
          const uint32_t lo = (uint32_t)(reinterpret_cast<uintptr_t>(src[a]) & 15);
          bulk_prefetch_l2(src[a] - lo, (lo + len[a] + 15) & ~15u);
        }
      };
      // results from staging back to global: the 16-byte-aligned interior by a
      // bulk copy, the few bytes before and after it by plain stores
      auto stage_out = [&](const unsigned char* s, float* g, uint32_t n) {
        const uintptr_t ga = reinterpret_cast<uintptr_t>(g);
        const uintptr_t a0 = (ga + 15) & ~uintptr_t(15), a1 = (ga + n) & ~uintptr_t(15);
        if (a1 > a0) bulk_s2g(reinterpret_cast<void*>(a0), saddr(s + (a0 - ga)), (uint32_t)(a1 - a0));
        const uintptr_t h1 = a1 > a0 ? a0 : ga + n;
        for (uintptr_t x = ga; x < h1; x += 4)
          *reinterpret_cast<float*>(x) = *reinterpret_cast<const float*>(s + (x - ga));
        if (a1 > a0)
          for (uintptr_t x = a1; x < ga + n; x += 4)
            *reinterpret_cast<float*>(x) = *reinterpret_cast<const float*>(s + (x - ga));
      };
      bool withhold = false;
      if (P.inject && (int)blockIdx.x < ntiles && *reinterpret_cast<volatile int*>(P.inject))
        withhold = atomicExch(P.inject, 0) != 0;
      bool mfail = false, issued = false;
      int loaded = -1;   // iteration whose staging loads are in flight / landed
      if ((int)blockIdx.x < ntiles) {
        stage_in(blockIdx.x);
        loaded = 0;
      }
      int it = 0;
      for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const uint32_t ph = it & 1;
        const int next = tile + gridDim.x;
        if (next < ntiles) prefetch(next);
        if (!mbar_wait(saddr(mbar + 1), ph)) { mfail = true; break; }
        fence_after();
        if constexpr (PML) {
          product(PL::cVF, PL::oAF, PL::SBF, PL::oBV, PL::SBF, NpK, idV);
          product(PL::cVP, PL::oAP, PL::SBF, PL::oBV, PL::SBF, NpK, idV);
        }
        product(PL::cD, PL::oAF, PL::SBF, PL::oBD, PL::SBF, NpK, idD);
        mma_commit(saddr(mbar + 3));
        issued = true;
        if (!mbar_wait(saddr(mbar + 2), ph)) { mfail = true; break; }
        fence_after();
        product(PL::cL, PL::oAL, PL::SBL, PL::oBL, PL::SBL, NFK, idL);
        if (!withhold) mma_commit(saddr(mbar + 4));
        withhold = false;
        if constexpr (PML) {
          if (!mbar_wait(saddr(mbar + 5), ph)) { mfail = true; break; }
          fence_after();
          product(PL::cVF, PL::oAF, PL::SBT, PL::oBP, PL::SBT, NqK, idP);
          product(PL::cVP, PL::oAP, PL::SBT, PL::oBP, PL::SBT, NqK, idP);
          mma_commit(saddr(mbar + 6));
        }
        if (!mbar_wait(saddr(mbar + 7), ph)) { mfail = true; break; }
        // results are staged in place of the inputs: write them back
        {
          int b, t0, ne;
          tile_geom(tile, b, t0, ne);
          const int64_t eg0 = P.e_begin + t0;
          const int64_t oq = (int64_t)b * P.strideQ + eg0 * 6 * Np;
          const int64_t op = (int64_t)b * P.strideP + (eg0 - P.K0) * 6 * Np;
          const uint32_t n = ne * 6 * Np * 4;
          stage_out(staged(PL::oSQ, P.qin + oq), P.qout + oq, n);
          stage_out(staged(PL::oSR, P.resq + oq), P.resq + oq, n);
          if constexpr (PML) {
            stage_out(staged(PL::oSP, P.p + op), P.p + op, n);
            stage_out(staged(PL::oSRP, P.resp + op), P.resp + op, n);
          }
          bulk_commit();
          bulk_wait_read();   // staging free for the next tile
        }
        if (next < ntiles) {
          stage_in(next);
          loaded = it + 1;
        }
      }
      // the staging copies in flight land before the memory is released
      if (loaded >= 0 && !mbar_wait(saddr(mbar + 0), loaded & 1)) mfail = true;
      bulk_wait_all();
      if (issued) {
        mma_commit(saddr(mbar + 8));
        if (!mbar_wait(saddr(mbar + 8), 0)) mfail = true;
      }
      if (mfail) atomicExch(P.err, 1);
    }
    __syncwarp();
  } else if (is_epilogue_warp<PL::QUADS>(warp)) {
    // ================================================= epilogue warps
    const int qd = warp & 3, h = warp >> 2;
    const int row = 32 * qd + lane;
    const int e = row >> 3, c = row & 7;
    const uint32_t tl = tmem + ((uint32_t)(32 * qd) << 16);   // this warp's lane quadrant
    // curl exchange partners (six live lanes of an element; pad lanes read
    // themselves): round 1 reads derivative (src+2)%3 of lane src1, round 2
    // derivative (src+1)%3 of lane src2
    constexpr int kSrc1[8] = {5, 3, 4, 2, 0, 1, 6, 7};
    constexpr int kSrc2[8] = {4, 5, 3, 1, 2, 0, 6, 7};
    const int base = lane & ~7;
    const int s1 = base + kSrc1[c], s2 = base + kSrc2[c];
    const int send1 = (c + 2) % 3, send2 = (c + 1) % 3;
    const int i0 = h * PL::NH, i1 = min(Np, i0 + PL::NH);   // nodes of this half
    int it = 0;
    for (int tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x, ++it) {
      const uint32_t ph = it & 1;
      int b, t0, ne;
      tile_geom(tile, b, t0, ne);
      const int64_t eg0 = P.e_begin + t0;
      const int64_t oq = (int64_t)b * P.strideQ + eg0 * 6 * Np;
      const int64_t op = (int64_t)b * P.strideP + (eg0 - P.K0) * 6 * Np;
      const bool live = c < 6 && e < ne;
      if (!mbar_wait(saddr(mbar + 0), ph)) { failed = true; break; }
      float* SQ = reinterpret_cast<float*>(staged(PL::oSQ, P.qin + oq));
      float* SR = reinterpret_cast<float*>(staged(PL::oSR, P.resq + oq));
      float* SP = PML ? reinterpret_cast<float*>(staged(PL::oSP, P.p + op)) : nullptr;
      float* SRP = PML ? reinterpret_cast<float*>(staged(PL::oSRP, P.resp + op)) : nullptr;
      // ---- A operands: this thread's row (e, c), its half of the K chunks
      {
        constexpr int NCH = NpK / CW;
        const int k0 = h ? (NCH + 1) / 2 : 0, k1 = h ? NCH : (NCH + 1) / 2;
        const float* fq = SQ + (e * 6 + c) * Np;
        const float* fp = PML ? SP + (e * 6 + c) * Np : nullptr;
        for (int kc = k0; kc < k1; ++kc) {
          float x[8], y[8];
#pragma unroll
          for (int u = 0; u < CW; ++u) {
            const int k = kc * CW + u;
            x[u] = live && k < Np ? fq[k] : 0.f;
            if constexpr (PML) y[u] = live && k < Np ? fp[k] : 0.f;
          }
          const uint32_t o = cofs<BF>(row, kc * CW, PL::SBF, 128);
          if constexpr (BF) {
            uint32_t w[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const __nv_bfloat162 v2 = __floats2bfloat162_rn(x[2 * u], x[2 * u + 1]);
              w[u] = *reinterpret_cast<const uint32_t*>(&v2);
            }
            *reinterpret_cast<uint4*>(smem + PL::oAF + o) = make_uint4(w[0], w[1], w[2], w[3]);
            if constexpr (PML) {
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const __nv_bfloat162 v2 = __floats2bfloat162_rn(y[2 * u], y[2 * u + 1]);
                w[u] = *reinterpret_cast<const uint32_t*>(&v2);
              }
              *reinterpret_cast<uint4*>(smem + PL::oAP + o) = make_uint4(w[0], w[1], w[2], w[3]);
            }
          } else {
            *reinterpret_cast<float4*>(smem + PL::oAF + o) =
                make_float4(to_tf32(x[0]), to_tf32(x[1]), to_tf32(x[2]), to_tf32(x[3]));
            if constexpr (PML)
              *reinterpret_cast<float4*>(smem + PL::oAP + o) =
                  make_float4(to_tf32(y[0]), to_tf32(y[1]), to_tf32(y[2]), to_tf32(y[3]));
          }
        }
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(saddr(mbar + 1));
      // this element's metric (r_x .. t_z) and 1/eps, 1/mu
      float g[9], ie = 0.f, im = 0.f;
      {
        const double* met = reinterpret_cast<const double*>(staged(PL::oSMET, P.geo + eg0 * 9));
        const float* mat = reinterpret_cast<const float*>(staged(PL::oSMAT, P.mat + eg0 * 3));
        const int ee = e < ne ? e : 0;
#pragma unroll
        for (int j = 0; j < 9; ++j) g[j] = (float)met[ee * 9 + j];
        ie = mat[ee * 3 + 0];
        im = mat[ee * 3 + 1];
      }
      if (!mbar_wait(saddr(mbar + 3), ph)) { failed = true; break; }
      fence_after();
      if constexpr (PML) {
        // ---- eq. 9 at this half's quadrature points -> T and Z rows
        const float* sg = reinterpret_cast<const float*>(
            staged(PL::oSSG, P.sig + (eg0 - P.K0) * 3 * NqP));
        const float ie0 = 1.f / (float)P.eps0;
        const int u = c % 3;
        const float* su_p = sg + (e * 3 + u) * NqP;
        const float* sv_p = sg + (e * 3 + (u + 1) % 3) * NqP;
        const float* sw_p = sg + (e * 3 + (u + 2) % 3) * NqP;
        const int q0 = h * PL::QH, q1 = min(NqK, q0 + PL::QH);
        for (int qq = q0; qq < q1; qq += 8) {
          // V_q of the F row and of the P row at points qq .. qq + 7
          float v[16];
          tld4x4(tl + PL::cVF + qq, tl + PL::cVP + qq, tl + PL::cVF + qq + 4,
                 tl + PL::cVP + qq + 4, v);
          float tz[2][8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int q = qq + j;
            const float vf = v[(j >> 2) * 8 + (j & 3)], vp = v[(j >> 2) * 8 + 4 + (j & 3)];
            float t = 0.f, z = 0.f;
            if (live && q < Nq && q < q1) {
              const float su = su_p[q] * ie0, sv = sv_p[q] * ie0, sw = sw_p[q] * ie0;
              // eq. 9 with kappa = 1 in terms of s = sigma / eps0:
              // b = sv + sw - su, c = sv sw - b su, d = su
              const float bc = sv + sw - su;
              const float cc = sv * sw - bc * su;
              t = bc * vf + cc * vp;
              z = vf - su * vp;
            }
            tz[0][j] = t;
            tz[1][j] = z;
          }
          // K chunks of CW points (4 TF32 / 8 BF16) of the T and Z rows
#pragma unroll
          for (int cj = 0; cj < 8 / CW; ++cj) {
            const int k = qq + cj * CW;
            if (k >= q1) break;
            const uint32_t o = cofs<BF>(row, k, PL::SBT, 128);
            if constexpr (BF) {
              uint32_t w0[4], w1[4];
#pragma unroll
              for (int u2 = 0; u2 < 4; ++u2) {
                const __nv_bfloat162 a2 = __floats2bfloat162_rn(tz[0][2 * u2], tz[0][2 * u2 + 1]);
                const __nv_bfloat162 b2 = __floats2bfloat162_rn(tz[1][2 * u2], tz[1][2 * u2 + 1]);
                w0[u2] = *reinterpret_cast<const uint32_t*>(&a2);
                w1[u2] = *reinterpret_cast<const uint32_t*>(&b2);
              }
              *reinterpret_cast<uint4*>(smem + PL::oAF + o) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
              *reinterpret_cast<uint4*>(smem + PL::oAP + o) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
            } else {
              const int j0 = cj * 4;
              *reinterpret_cast<float4*>(smem + PL::oAF + o) =
                  make_float4(to_tf32(tz[0][j0]), to_tf32(tz[0][j0 + 1]), to_tf32(tz[0][j0 + 2]),
                              to_tf32(tz[0][j0 + 3]));
              *reinterpret_cast<float4*>(smem + PL::oAP + o) =
                  make_float4(to_tf32(tz[1][j0]), to_tf32(tz[1][j0 + 1]), to_tf32(tz[1][j0 + 2]),
                              to_tf32(tz[1][j0 + 3]));
            }
          }
        }
        fence_async_smem();
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(saddr(mbar + 5));
      }
      // ---- curl with the LIFT term: right-hand side of E, H at this half's
      // nodes, kept in registers until the update
      if (!mbar_wait(saddr(mbar + 4), ph)) { failed = true; break; }
      fence_after();
      constexpr int NHC = PL::NH;
      float rhs[NHC];
      const int eg = (int)eg0 + (e < ne ? e : 0);
#pragma unroll
      for (int ic = 0; ic < NHC; ic += 4) {
        const int i = i0 + ic;
        float v[16];   // d/dr, d/ds, d/dt, LIFT at nodes i .. i + 3
        tld4x4(tl + PL::cD + i, tl + PL::cD + NpA + i, tl + PL::cD + 2 * NpA + i, tl + PL::cL + i,
               v);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float dr = v[j], ds = v[4 + j], dt = v[8 + j], lf = v[12 + j];
          const float d[3] = {g[0] * dr + g[3] * ds + g[6] * dt, g[1] * dr + g[4] * ds + g[7] * dt,
                              g[2] * dr + g[5] * ds + g[8] * dt};
          const float a1 = __shfl_sync(0xffffffffu, d[send1], s1);
          const float a2 = __shfl_sync(0xffffffffu, d[send2], s2);
          const float cr = a1 - a2 + lf;   // (curl of the partner field) + LIFT term
          rhs[ic + j] = c < 3 ? ie * cr : -im * cr;
        }
      }
      // dipole sources of this element (E rows): -J(t) dir M_k^-1 l(r_s)
      if (live && c < 3) {
        for (int s = 0; s < P.nsrc; ++s) {
          const int sb = s < kSrcCache ? srcc[2 * s] : P.src[s].batch;
          const int se = s < kSrcCache ? srcc[2 * s + 1] : P.src[s].elem;
          if (sb != b || se != eg) continue;
          const SrcDev& sd = P.src[s];
          const double tau = sd.width;
          const double gg = exp(-(tst - sd.t0) * (tst - sd.t0) / (4.0 * tau * tau));
          const float jt = (float)(sd.amp * (-(tst - sd.t0) / (2.0 * tau * tau)) * gg) *
                           (float)sd.dir[c];
#pragma unroll
          for (int ic = 0; ic < NHC; ++ic)
            if (i0 + ic < i1) rhs[ic] -= ie * jt * P.src_w[s * Np + i0 + ic];
        }
      }
      if constexpr (PML) {
        if (!mbar_wait(saddr(mbar + 6), ph)) { failed = true; break; }
        fence_after();
      }
      // ---- Runge-Kutta update of this half's nodes, in place in the staging
#pragma unroll
      for (int ic = 0; ic < NHC; ic += 4) {
        const int i = i0 + ic;
        float sz[8];   // s (E, H row) | rhs of P (P row) at nodes i .. i + 3
        if constexpr (PML) {
          tld4x2(tl + PL::cVF + i, tl + PL::cVP + i, sz);
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j) sz[j] = 0.f;
        }
        if (!live) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int ii = i + j;
          if (ii >= i1) break;
          const int li = (e * 6 + c) * Np + ii;
          const float rr = rka * SR[li] + rdt * (rhs[ic + j] - sz[j]);
          SR[li] = rr;
          SQ[li] = SQ[li] + rkb * rr;
          if constexpr (PML) {
            const float rp = rka * SRP[li] + rdt * sz[4 + j];
            SRP[li] = rp;
            SP[li] = SP[li] + rkb * rp;
          }
        }
      }
      fence_async_smem();   // the bulk copies read these values
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(saddr(mbar + 7));
    }
    if (failed && lane == 0) atomicExch(P.err, 1);
  } else {
    // ================================================= flux warps
    int fw = 0;   // index among the flux warps
    for (int w = 0; w < warp; ++w) fw += !is_epilogue_warp<PL::QUADS>(w) && w < 12;
    const int ft = fw * 32 + lane;   // flux thread
    constexpr int NFT = 32 * PL::NFW;
    int it = 0;
    for (int tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x, ++it) {
      const uint32_t ph = it & 1;
      int b, t0, ne;
      tile_geom(tile, b, t0, ne);
      const int64_t eg0 = P.e_begin + t0;
      const int64_t oq = (int64_t)b * P.strideQ + eg0 * 6 * Np;
      const float* qin = P.qin + (int64_t)b * P.strideQ;
      // neighbour ids and traces first (global memory), then the own traces
      constexpr int FT = (T * NF + NFT - 1) / NFT;
      float Ep[FT][3], Hp[FT][3], ZPv[FT];
#pragma unroll
      for (int u = 0; u < FT; ++u) {
        const int task = ft + u * NFT;
        ZPv[u] = -1.f;
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) { Ep[u][cc] = 0.f; Hp[u][cc] = 0.f; }
        if (task < ne * NF) {
          const int e = task / NF, fm = task - e * NF, f = fm / Nfp, m = fm - f * Nfp;
          const int nb = P.nbr[(eg0 + e) * 4 + f];
          if (nb >= 0) {
            const int code = P.code[(eg0 + e) * 4 + f];
            if (!WADG_INDEX_OK(nb < P.strideQ / (6 * Np) && code < 24, P.err)) continue;
            const int np2 = fperm[(f * 24 + code) * Nfp + m];
            if (!WADG_INDEX_OK(np2 < Np, P.err)) continue;
            const float* qn = qin + (int64_t)nb * 6 * Np + np2;
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) { Ep[u][cc] = qn[cc * Np]; Hp[u][cc] = qn[(3 + cc) * Np]; }
            ZPv[u] = P.mat[nb * 3 + 2];
          }
        }
      }
      if (!mbar_wait(saddr(mbar + 0), ph)) { failed = true; break; }
      const float* SQ = reinterpret_cast<const float*>(staged(PL::oSQ, P.qin + oq));
      const float* fn_s = reinterpret_cast<const float*>(staged(PL::oSFN, P.fnrm + eg0 * 16));
      const float* mat_s = reinterpret_cast<const float*>(staged(PL::oSMAT, P.mat + eg0 * 3));
      const float al = (float)P.alpha;
#pragma unroll
      for (int u = 0; u < FT; ++u) {
        const int task = ft + u * NFT;
        if (task >= ne * NF) continue;
        const int e = task / NF, fm = task - e * NF, f = fm / Nfp;
        const int ni = Fmask[fm];
        const float* nn = fn_s + e * 16 + f * 4;
        const float nx = nn[0], ny = nn[1], nz = nn[2], fsc = nn[3];
        const float* sq = SQ + e * 6 * Np + ni;
        float Em[3], Hm[3], Eo[3], Ho[3];
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) { Em[cc] = sq[cc * Np]; Hm[cc] = sq[(3 + cc) * Np]; }
        const float ZM = mat_s[e * 3 + 2];
        float ZP = ZPv[u];
        if (ZP < 0.f) {   // perfect electric conductor: mirror state
          ZP = ZM;
#pragma unroll
          for (int cc = 0; cc < 3; ++cc) { Eo[cc] = -Em[cc]; Ho[cc] = Hm[cc]; }
        } else {
#pragma unroll
          for (int cc = 0; cc < 3; ++cc) { Eo[cc] = Ep[u][cc]; Ho[cc] = Hp[u][cc]; }
        }
        const float dEx = Eo[0] - Em[0], dEy = Eo[1] - Em[1], dEz = Eo[2] - Em[2];
        const float dHx = Ho[0] - Hm[0], dHy = Ho[1] - Hm[1], dHz = Ho[2] - Hm[2];
        const float ndE = nx * dEx + ny * dEy + nz * dEz;
        const float ndH = nx * dHx + ny * dHy + nz * dHz;
        const float cHx = ny * dHz - nz * dHy, cHy = nz * dHx - nx * dHz, cHz = nx * dHy - ny * dHx;
        const float cEx = ny * dEz - nz * dEy, cEy = nz * dEx - nx * dEz, cEz = nx * dEy - ny * dEx;
        const float YM = __fdividef(1.f, ZM), YP = __fdividef(1.f, ZP);
        const float sH = __fdividef(fsc, ZM + ZP), sE = __fdividef(fsc, YM + YP);
        float fo[6];
        fo[0] = sH * (ZP * cHx - al * (nx * ndE - dEx));
        fo[1] = sH * (ZP * cHy - al * (ny * ndE - dEy));
        fo[2] = sH * (ZP * cHz - al * (nz * ndE - dEz));
        fo[3] = sE * (YP * cEx + al * (nx * ndH - dHx));
        fo[4] = sE * (YP * cEy + al * (ny * ndH - dHy));
        fo[5] = sE * (YP * cEz + al * (nz * ndH - dHz));
#pragma unroll
        for (int cc = 0; cc < 6; ++cc)
          put_op<BF>(smem + PL::oAL + cofs<BF>(8 * e + cc, fm, PL::SBL, 128), fo[cc]);
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(saddr(mbar + 2));
    }
    if (failed && lane == 0) atomicExch(P.err, 1);
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) tmem_dealloc(tmem, PL::TMEM_COLS);
  (void)nqd;
}

template <int N, bool PML, bool BF>
cudaError_t rows_configure() {
  return cudaFuncSetAttribute(tc_rows_kernel<N, PML, BF>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)RPlan<N, PML, BF>::bytes);
}

template <int N, bool PML, bool BF>
cudaError_t rows_launch(const StageParams<float>& P, int nb, cudaStream_t s) {
  using PL = RPlan<N, PML, BF>;
  if (P.n_elem <= 0) return cudaSuccess;
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  StageParams<float> Q = P;
  Q.nb = nb;
  const long long tiles = (long long)((P.n_elem + PL::T - 1) / PL::T) * nb;
  const int grid = (int)std::min<long long>(tiles, (long long)sms);
  tc_rows_kernel<N, PML, BF><<<grid, PL::THREADS, PL::bytes, s>>>(Q);
  return cudaGetLastError();
}

}  // namespace tc

template <bool BF>
cudaError_t configure_rows_bf(int N) {
  switch (N) {
    case 1: return tc::rows_configure<1, true, BF>();
    case 2: return tc::rows_configure<2, true, BF>();
    case 3: return tc::rows_configure<3, true, BF>();
    case 4: return tc::rows_configure<4, true, BF>();
    case 5: return tc::rows_configure<5, true, BF>();
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t configure_tc_rows(int N, bool bf16) {
  return bf16 ? configure_rows_bf<true>(N) : configure_rows_bf<false>(N);
}

template <bool BF>
cudaError_t launch_rows_bf(int N, const StageParams<float>& P, int nb, cudaStream_t s) {
  switch (N) {
    case 1: return tc::rows_launch<1, true, BF>(P, nb, s);
    case 2: return tc::rows_launch<2, true, BF>(P, nb, s);
    case 3: return tc::rows_launch<3, true, BF>(P, nb, s);
    case 4: return tc::rows_launch<4, true, BF>(P, nb, s);
    case 5: return tc::rows_launch<5, true, BF>(P, nb, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_pml_tc_rows(int N, const StageParams<float>& P, int nb, cudaStream_t s,
                               bool bf16) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(P.qin) | reinterpret_cast<uintptr_t>(P.qout) |
                      reinterpret_cast<uintptr_t>(P.resq) | reinterpret_cast<uintptr_t>(P.p) |
                      reinterpret_cast<uintptr_t>(P.resp) | reinterpret_cast<uintptr_t>(P.sig);
  if (a & 15) return cudaErrorMisalignedAddress;
  return bf16 ? launch_rows_bf<true>(N, P, nb, s) : launch_rows_bf<false>(N, P, nb, s);
}

}  // namespace wadg
