// Tensor-core stage kernel with row-owned epilogues (sm_103a: tcgen05 with
// TF32 or BF16 operands, FP32 accumulation in tensor memory, FP32 state) for
// the PML class of contexts with a compact volume rule (quad_capacity class
// 1).  The kernel is written for both element classes (PML = false drops the
// P rows, V_q, P_q and eq. 9), but only the PML class is built: at N = 4 the
// non-PML instantiation took 0.376 ms per launch (TF32) against 0.342 ms for
// the non-PML class of tc_stage_kernel, which keeps that class.
//
// Every contraction of the stage is one product
//     D[row][n] = sum_k A[row][k] * B[n][k]
// whose A operand is the tile's field data, one row per (element,
// component), and whose B operand is the reference operator (row n = output
// node, quadrature point or stacked derivative).  A tile is 8 elements of 8
// rows each (Ex, Ey, Ez, Hx, Hy, Hz and two zero rows): 64 of the M = 128
// rows of a product, and so 64 of the 128 tensor-memory lanes.  A block runs
// two tiles at once ("slots", each with its own buffers, columns and issuing
// thread; one when a slot needs more than half of the tensor memory): slot
// 0's rows are lanes 0-63 and slot 1's lanes 64-127, its products starting 8
// row groups before its operand buffers.  The thread that owns lane (e, c)
// receives every output of every product for its element and component:
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
// Warp roles per slot: four epilogue warps (two per lane quadrant of the
// slot, splitting the nodes and quadrature points of their rows in halves),
// flux warps (upwind flux into the LIFT operand) and an issuing warp whose
// first lane stages each tile with bulk copies (and prefetches the next tile
// into L2), issues every product and writes the results back with bulk
// copies.  Every wait is bounded; on timeout the kernel records an
// error, drains its copies and products and releases its tensor memory.
#include "kernels.cuh"
#include "tc_ptx.cuh"

#include <algorithm>
#include <cstdint>
#include <type_traits>

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
  static constexpr int T = 8;                       // elements per tile (slot)
  static constexpr int NpA = rup4(Np);              // stacked derivative block
  // product widths (columns): V_q, stacked derivatives, LIFT, P_q
  static constexpr int NV = rup16(Nq), ND = rup16(3 * NpA), NL = rup16(Np), NPQ = rup16(Np);
  static_assert(NPQ <= NV, "P_q outputs reuse the V_q columns");
  static_assert(NV <= 256 && ND <= 256, "product width");
  // tensor-memory columns of one slot
  static constexpr uint32_t cVF = 0, cVP = PML ? NV : 0;
  static constexpr uint32_t cD = PML ? 2 * NV : 0, cL = cD + ND;
  static constexpr uint32_t COLS = cL + NL;
  static constexpr uint32_t pow2(uint32_t c) {
    return c <= 32 ? 32 : c <= 64 ? 64 : c <= 128 ? 128 : c <= 256 ? 256 : 512;
  }
  // two slots (two tiles in flight, one per half of the lanes) when each
  // fits half of the tensor memory, else one
  static constexpr int SLOTS = pow2(COLS) <= 256 ? 2 : 1;
  static constexpr uint32_t CSTR = pow2(COLS);      // column stride between slots
  static constexpr uint32_t TMEM_COLS = SLOTS * CSTR;
  static_assert(TMEM_COLS <= 512, "tensor-memory columns");
  // canonical K-major layout without swizzle: 8-row x 16-byte core matrices,
  // K-adjacent core matrices 128 bytes apart, 8-row groups SB(K) apart
  __host__ __device__ static constexpr uint32_t SB(int K) { return (uint32_t)(K / CW) * 128u; }
  static constexpr uint32_t SBF = SB(NpK), SBT = SB(NqK), SBL = SB(NFK);
  // the flux operand (A of LIFT) is written one face node (K) per lane: a
  // 144-byte step between K-adjacent core matrices puts a warp's 32
  // consecutive K on distinct banks (128 bytes puts them on four banks: 8-way
  // conflicts for TF32, 4-way for BF16, whose lanes share words)
  static constexpr uint32_t LBA = 144, SBLA = (uint32_t)(NFK / CW) * LBA;
  // B operands (the reference operators, staged once per block)
  static constexpr uint32_t oBD = 0;
  static constexpr uint32_t oBL = oBD + (ND / 8) * SBF;
  static constexpr uint32_t oBV = oBL + (NL / 8) * SBL;
  static constexpr uint32_t oBP = oBV + (PML ? (NV / 8) * SBF : 0);
  static constexpr uint32_t oA = oBP + (PML ? (NPQ / 8) * SBT : 0);
  // A operands of a slot (8 element rows groups each): F then T, P then Z,
  // flux.  A product reads 128 rows: slot 0's live rows are rows 0-63 (the
  // rest fall on the buffers after), slot 1's product starts 8 row groups
  // before its buffers so that its live rows are rows 64-127 (lanes 64-127)
  static constexpr uint32_t AFB = 8 * (PML && SBT > SBF ? SBT : SBF);
  static constexpr uint32_t oAF = 0, oAP = AFB, oAL = oAP + (PML ? AFB : 0);
  static constexpr uint32_t ASLOT = oAL + 8 * SBLA;
  // staging of a slot, each block copied as the 16-byte-aligned cover of its
  // data.  Early blocks (E,H, P, geometry, neighbour tables: needed from the
  // start of a tile, the tables by the flux warps one tile earlier)
  // have EB buffers, so the next tile's land while this one computes; late
  // blocks (the Runge-Kutta registers, needed at the update, and the sigma
  // samples, needed at eq. 9) have one, refilled once this tile is past them.
  static constexpr uint32_t FB = ((T * 6 * Np * 4 + 15) & ~15) + 16;
  static constexpr uint32_t SGB = PML ? ((T * 3 * NqP * 4 + 15) & ~15) + 16 : 0;
  static constexpr uint32_t GFN = ((T * 64 + 15) & ~15) + 16;
  static constexpr uint32_t GMET = ((T * 72 + 15) & ~15) + 16;
  static constexpr uint32_t GMAT = ((T * 12 + 15) & ~15) + 16;
  static constexpr uint32_t oEQ = 0, oEP = FB, oEFN = oEP + (PML ? FB : 0);
  static constexpr uint32_t oEMET = oEFN + GFN, oEMAT = oEMET + GMET;
  // the tile's face neighbours (int) and orientation codes (byte), [T][4]
  static constexpr uint32_t GNB = ((T * 16 + 15) & ~15) + 16, GCD = ((T * 4 + 15) & ~15) + 16;
  static constexpr uint32_t oENB = oEMAT + GMAT, oECD = oENB + GNB;
  static constexpr uint32_t EBUF = (oECD + GCD + 127) & ~127u;   // one early buffer
  static constexpr uint32_t oLR = 0, oLRP = FB, oLSG = oLRP + (PML ? FB : 0);
  static constexpr uint32_t LBUF = (oLSG + SGB + 127) & ~127u;     // the late buffer
  __host__ __device__ static constexpr uint32_t misc_bytes() {
    return 256 + 16 + 512 + ((100 * Nfp + 15) & ~15u);
  }
  __host__ __device__ static constexpr uint32_t total(int eb) {
    return oA + SLOTS * ASLOT + SLOTS * (eb * EBUF + LBUF) + misc_bytes();
  }
  static constexpr int EB = total(2) <= 227 * 1024 ? 2 : 1;
  static constexpr uint32_t SSLOT = EB * EBUF + LBUF;
  static constexpr uint32_t oST = oA + SLOTS * ASLOT;
  static constexpr uint32_t oMisc = oST + SLOTS * SSLOT;
  // misc: 2 x 12 mbarriers | TMEM slot | cached sources (64 x (batch,
  // element)) | face tables (Fmask [NF], fperm [4][24][Nfp])
  static constexpr uint32_t oTabs = 256 + 16 + 512;
  static constexpr uint32_t bytes_used = oMisc + misc_bytes();
  // a block holding all 512 tensor-memory columns asks for more than half the
  // shared memory, so that no second block can wait in tcgen05.alloc
  static constexpr uint32_t bytes =
      TMEM_COLS == 512 && bytes_used < 116 * 1024 ? 116 * 1024 : bytes_used;
  // every product's 128-row read stays inside the block: slot 0 reads from
  // its buffers on, slot 1 from 8 row groups before them
  __host__ __device__ static constexpr bool span_ok(uint32_t o, uint32_t sb) {
    return oA + o + 16 * sb <= bytes &&
           (SLOTS == 1 || (oA + ASLOT + o >= 8 * sb && oA + ASLOT + o + 8 * sb <= bytes));
  }
  static_assert(span_ok(oAF, SBF) && span_ok(oAL, SBLA), "F / flux operand span");
  static_assert(!PML || (span_ok(oAP, SBF) && span_ok(oAF, SBT) && span_ok(oAP, SBT)),
                "P / T / Z operand span");
  static_assert(bytes <= 227 * 1024, "shared memory");
  // warps: 4 epilogue warps per slot (the two lane quadrants of the slot x
  // halves of the nodes and points), flux warps, an issuing warp and a copy
  // warp per slot
  // S epilogue warps per lane quadrant, each taking a share of the nodes
  // and quadrature points of the quadrant's rows
  static constexpr int S = 2;
  static constexpr int EW = 4 * S;                  // warps 0 .. EW-1: epilogue / flux
  static constexpr int FLUXW = SLOTS == 2 ? 2 : 2 * S + 4;   // flux warps per slot
  // warps: EW epilogue (and, with one slot, flux), 4 flux, then one issuing
  // warp and one copy warp per slot
  static constexpr int THREADS = 32 * (EW + 4 + 2 * SLOTS);
  // nodes and quadrature points of one split (multiples of 4)
  // register split (two slots: the warp groups are 0-7 epilogue, 8-11
  // flux, 12-15 issuing and copy): setmaxnreg moves registers from the flux
  // and copy groups to the epilogue warps within the launch allocation
  static constexpr int LAUNCH_REGS = (65536 / THREADS) & ~7;
  static constexpr int REG_E = 128, REG_F = 96, REG_C = 96;
  static constexpr bool SPLIT = false;   // measured: the uniform budget is faster
  static_assert(!SPLIT || 32 * (EW * REG_E + 4 * REG_F + 4 * REG_C) <= THREADS * LAUNCH_REGS,
                "register split within the launch allocation");
  static constexpr int NS = rup4((Np + S - 1) / S);
  static constexpr int QS = ((NqK / CW + S - 1) / S) * CW;
  static_assert(QS % 4 == 0, "quadrature split");
};

// warp roles.  Epilogue warps: w < EW whose lane quadrant w & 3 belongs to
// a slot (quadrants 0, 1 -> slot 0; 2, 3 -> slot 1 when there are two).
// Flux warps: the other warps below EW + 4.  Then the issuing warps
// (EW + 4 + slot) and the copy warps (EW + 4 + SLOTS + slot).
template <int SLOTS, int EW>
__device__ __forceinline__ int epilogue_slot(int w) {
  if (w >= EW) return -1;
  const int qd = w & 3;
  if (SLOTS == 2) return qd >> 1;
  return qd < 2 ? 0 : -1;
}
template <int SLOTS, int EW>
__device__ __forceinline__ int flux_slot(int w, int& index) {
  if (SLOTS == 2) {   // warps EW .. EW + 3: two per slot
    if (w < EW || w >= EW + 4) return -1;
    index = (w - EW) & 1;
    return (w - EW) >> 1;
  }
  // one slot: the warps of quadrants 2 and 3 below EW, then EW .. EW + 3
  if (w >= EW + 4 || epilogue_slot<1, EW>(w) >= 0) return -1;
  index = w < EW ? (w >> 2) * 2 + (w & 1) : EW / 2 + (w - EW);
  return 0;
}

template <int N, bool PML, bool BF>
__global__ void __launch_bounds__(RPlan<N, PML, BF>::THREADS, 1)
    tc_rows_kernel(const StageParams<float> P) {
  using PL = RPlan<N, PML, BF>;
  constexpr int Np = PL::Np, Nfp = PL::Nfp, NF = PL::NF, Nq = PL::Nq, T = PL::T;
  constexpr int NpK = PL::NpK, NFK = PL::NFK, NqK = PL::NqK, CW = PL::CW, KS = PL::KS;
  constexpr int NpA = PL::NpA, NqP = PL::NqP, SLOTS = PL::SLOTS, EB = PL::EB;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t sbase = saddr(smem);
  // mbarriers of slot s at mbar + 12 s: [0], [1] early buffer 0 / 1 landed,
  // [2] late registers landed, [3] sigma landed, [4] F/P operands ready,
  // [5] flux ready, [6] V_q and derivative products done (the F and P
  // operands are free), [7] derivative and LIFT products done, [8] T/Z
  // ready, [9] P_q done, [10] results staged, [11] final drain
  enum { B_E0 = 0, B_LATE = 2, B_SIG = 3, B_FP = 4, B_FLUX = 5, B_V = 6, B_L = 7, B_TZ = 8,
         B_PQ = 9, B_OUT = 10, B_DRAIN = 11 };
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + PL::oMisc);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + PL::oMisc + 256);
  int* srcc = reinterpret_cast<int*>(smem + PL::oMisc + 272);   // [64][2]
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
    constexpr uint32_t ne_ = 2 * PL::S;   // epilogue warps per slot
    const uint32_t cnt[12] = {1, 1, 1, 1, ne_, (uint32_t)PL::FLUXW, 1, 1, ne_, 1, ne_, 1};
    for (int sl = 0; sl < SLOTS; ++sl)
      for (int i = 0; i < 12; ++i) mbar_init(saddr(mbar + 12 * sl + i), cnt[i]);
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
  // tiles of slot s: worker blockIdx.x * SLOTS + s of gridDim.x * SLOTS
  const int nworkers = gridDim.x * SLOTS;
  bool failed = false;

  struct Tile {
    int b, ne;
    int64_t eg0, oq, op;
  };
  auto tile_at = [&](int tile) {
    Tile t;
    t.b = tile / tiles_per_batch;
    const int t0 = (tile - t.b * tiles_per_batch) * T;
    t.ne = min(T, P.n_elem - t0);
    t.eg0 = P.e_begin + t0;
    t.oq = (int64_t)t.b * P.strideQ + t.eg0 * 6 * Np;
    t.op = (int64_t)t.b * P.strideP + (t.eg0 - P.K0) * 6 * Np;
    return t;
  };
  // where the first value of a staged block lands (its cover starts at the
  // 16-byte boundary below it)
  auto staged = [&](uint32_t o, const void* g) {
    return smem + o + (reinterpret_cast<uintptr_t>(g) & 15);
  };
  auto ebuf = [&](int sl, int it) {   // early buffer of iteration it
    return PL::oST + sl * PL::SSLOT + (EB == 2 ? (it & 1) : 0) * PL::EBUF;
  };
  auto lbuf = [&](int sl) { return PL::oST + sl * PL::SSLOT + EB * PL::EBUF; };
  // phase parity of early buffer (it & 1) at iteration it
  auto eparity = [&](int it) { return (uint32_t)(EB == 2 ? (it >> 1) & 1 : it & 1); };

  if (warp >= PL::EW + 4) {
    if constexpr (PL::SPLIT) asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(PL::REG_C));
    // ================================ issuing and copy warps of a slot (lane 0)
    const bool copier = warp >= PL::EW + 4 + SLOTS;
    const int sl = warp - PL::EW - 4 - (copier ? SLOTS : 0);
    const uint32_t sA = PL::oA + sl * PL::ASLOT;      // this slot's A operands
    uint64_t* mb = mbar + 12 * sl;
    const uint32_t tcol = tmem + sl * PL::CSTR;       // this slot's columns, lane 0
    const int first = blockIdx.x * SLOTS + sl;
    if (lane == 0 && !copier) {
      // ---------------------------------------------- products
      constexpr uint32_t idV = BF ? idesc_bf16(128, PL::NV) : idesc_tf32(128, PL::NV);
      constexpr uint32_t idD = BF ? idesc_bf16(128, PL::ND) : idesc_tf32(128, PL::ND);
      constexpr uint32_t idL = BF ? idesc_bf16(128, PL::NL) : idesc_tf32(128, PL::NL);
      constexpr uint32_t idP = BF ? idesc_bf16(128, PL::NPQ) : idesc_tf32(128, PL::NPQ);
      auto mma = [](uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
        if constexpr (BF) mma_bf16(d, a, b, id, acc);
        else mma_tf32(d, a, b, id, acc);
      };
      // D[col] = A (buffer aoff of this slot, row-group stride sba) x B^T; slot
      // 1 starts 8 row groups before its buffer (its rows are lanes 64-127)
      auto product = [&](uint32_t col, uint32_t aoff, uint32_t sba, uint32_t boff, uint32_t sbb,
                         int K, uint32_t id) {
        const uint32_t a0 = sbase + sA + aoff - (sl ? 8 * sba : 0);
        const uint32_t lba = aoff == PL::oAL ? PL::LBA : 128u;
        for (int k = 0; k < K / KS; ++k)
          mma(tcol + col, make_desc(a0 + 2 * lba * k, lba, sba),
              make_desc(sbase + boff + 256 * k, 128, sbb), id, k > 0);
      };
      bool withhold = false;
      if (P.inject && first < ntiles && *reinterpret_cast<volatile int*>(P.inject))
        withhold = atomicExch(P.inject, 0) != 0;
      bool mfail = false, issued = false;
      int it = 0;
      for (int tile = first; tile < ntiles; tile += nworkers, ++it) {
        const uint32_t ph = it & 1;
        if (!mbar_wait_sleep(saddr(mb + B_FP), ph)) { mfail = true; break; }
        fence_after();
        issued = true;
        if constexpr (PML) {   // V_q first, then the derivatives
          product(PL::cVF, PL::oAF, PL::SBF, PL::oBV, PL::SBF, NpK, idV);
          product(PL::cVP, PL::oAP, PL::SBF, PL::oBV, PL::SBF, NpK, idV);
        }
        product(PL::cD, PL::oAF, PL::SBF, PL::oBD, PL::SBF, NpK, idD);
        // eq. 9 writes its T and Z rows over the F and P operands: it waits
        // until every product reading them (V_q and the derivatives) is done
        if constexpr (PML) mma_commit(saddr(mb + B_V));
        if (!mbar_wait_sleep(saddr(mb + B_FLUX), ph)) { mfail = true; break; }
        fence_after();
        product(PL::cL, PL::oAL, PL::SBLA, PL::oBL, PL::SBL, NFK, idL);
        if (!withhold) mma_commit(saddr(mb + B_L));   // derivatives and LIFT
        withhold = false;
        if constexpr (PML) {
          if (!mbar_wait_sleep(saddr(mb + B_TZ), ph)) { mfail = true; break; }
          fence_after();
          product(PL::cVF, PL::oAF, PL::SBT, PL::oBP, PL::SBT, NqK, idP);
          product(PL::cVP, PL::oAP, PL::SBT, PL::oBP, PL::SBT, NqK, idP);
          mma_commit(saddr(mb + B_PQ));
        }
      }
      // every product this thread issued completes before the memory is released
      if (issued) {
        mma_commit(saddr(mb + B_DRAIN));
        if (!mbar_wait_sleep(saddr(mb + B_DRAIN), 0)) mfail = true;
      }
      if (mfail) atomicExch(P.err, 1);
    } else if (lane == 0) {
      // ---------------------------------------------- staging copies
      // bulk copies of global blocks (16-byte-aligned covers) into staging,
      // completing on barrier `bar`
      auto copy_in = [&](const void* const* src, const uint32_t* len, const uint32_t* dst, int n,
                         uint64_t* bar) {
        uint32_t total = 0;
        for (int a = 0; a < n; ++a) {
          const uint32_t lo = (uint32_t)(reinterpret_cast<uintptr_t>(src[a]) & 15);
          total += (lo + len[a] + 15) & ~15u;
        }
        fence_async_smem();
        mbar_expect_tx(saddr(bar), total);
        for (int a = 0; a < n; ++a) {
          const uint32_t lo = (uint32_t)(reinterpret_cast<uintptr_t>(src[a]) & 15);
          bulk_g2s(sbase + dst[a], static_cast<const unsigned char*>(src[a]) - lo,
                   (lo + len[a] + 15) & ~15u, saddr(bar));
        }
      };
      auto early_in = [&](int tile, int it) {
        const Tile t = tile_at(tile);
        const uint32_t eb = ebuf(sl, it), fb = t.ne * 6 * Np * 4;
        const void* src[7] = {P.qin + t.oq, PML ? (const void*)(P.p + t.op) : nullptr,
                              P.fnrm + t.eg0 * 16, P.geof + t.eg0 * 9, P.mat + t.eg0 * 3,
                              P.nbr + t.eg0 * 4, P.code + t.eg0 * 4};
        const uint32_t len[7] = {fb, fb, (uint32_t)t.ne * 64, (uint32_t)t.ne * 36,
                                 (uint32_t)t.ne * 12, (uint32_t)t.ne * 16, (uint32_t)t.ne * 4};
        const uint32_t dst[7] = {eb + PL::oEQ, eb + PL::oEP, eb + PL::oEFN, eb + PL::oEMET,
                                 eb + PL::oEMAT, eb + PL::oENB, eb + PL::oECD};
        // the neighbour tables travel with the early blocks when there are two
        // early buffers (the flux warps read them a tile ahead)
        constexpr int NBK = EB == 2 ? 7 : 5;
        if constexpr (PML) {
          copy_in(src, len, dst, NBK, mb + B_E0 + (EB == 2 ? (it & 1) : 0));
        } else {
          const void* s2[6] = {src[0], src[2], src[3], src[4], src[5], src[6]};
          const uint32_t l2[6] = {len[0], len[2], len[3], len[4], len[5], len[6]};
          const uint32_t d2[6] = {dst[0], dst[2], dst[3], dst[4], dst[5], dst[6]};
          copy_in(s2, l2, d2, NBK - 1, mb + B_E0 + (EB == 2 ? (it & 1) : 0));
        }
      };
      auto late_in = [&](int tile) {
        const Tile t = tile_at(tile);
        const uint32_t lb = lbuf(sl), fb = t.ne * 6 * Np * 4;
        const void* src[2] = {P.resq + t.oq, PML ? (const void*)(P.resp + t.op) : nullptr};
        const uint32_t len[2] = {fb, fb};
        const uint32_t dst[2] = {lb + PL::oLR, lb + PL::oLRP};
        copy_in(src, len, dst, PML ? 2 : 1, mb + B_LATE);
      };
      auto sig_in = [&](int tile) {
        if constexpr (PML) {
          const Tile t = tile_at(tile);
          const void* src[1] = {P.sig + (t.eg0 - P.K0) * 3 * NqP};
          const uint32_t len[1] = {(uint32_t)t.ne * 3 * NqP * 4};
          const uint32_t dst[1] = {lbuf(sl) + PL::oLSG};
          copy_in(src, len, dst, 1, mb + B_SIG);
        }
      };
      auto prefetch = [&](int tile) {
        const Tile t = tile_at(tile);
        const uint32_t fb = t.ne * 6 * Np * 4;
        const void* src[8] = {P.qin + t.oq, P.resq + t.oq, P.fnrm + t.eg0 * 16, P.geof + t.eg0 * 9,
                              P.mat + t.eg0 * 3, PML ? (const void*)(P.p + t.op) : nullptr,
                              PML ? (const void*)(P.resp + t.op) : nullptr,
                              PML ? (const void*)(P.sig + (t.eg0 - P.K0) * 3 * NqP) : nullptr};
        const uint32_t len[8] = {fb, fb, (uint32_t)t.ne * 64, (uint32_t)t.ne * 36,
                                 (uint32_t)t.ne * 12, fb, fb, (uint32_t)t.ne * 3 * NqP * 4};
        for (int a = 0; a < (PML ? 8 : 5); ++a) {
          const uint32_t lo = (uint32_t)(reinterpret_cast<uintptr_t>(src[a]) & 15);
          bulk_prefetch_l2(static_cast<const unsigned char*>(src[a]) - lo,
                           (lo + len[a] + 15) & ~15u);
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
      bool cfail = false;
      // in-flight copies to drain on exit: last iteration of each kind
      int pend_e[2] = {-1, -1}, pend_l = -1, pend_s = -1;
      if (first < ntiles) {
        early_in(first, 0);
        pend_e[0] = 0;
        late_in(first);
        pend_l = 0;
        sig_in(first);
        pend_s = 0;
      }
      int it = 0;
      for (int tile = first; tile < ntiles; tile += nworkers, ++it) {
        const uint32_t ph = it & 1;
        const int next = tile + nworkers;
        // the next tile's early blocks into the other buffer (its previous
        // tile's results were written back at the end of the last iteration)
        if (EB == 2 && next < ntiles) {
          early_in(next, it + 1);
          pend_e[(it + 1) & 1] = it + 1;
        }
        if (next + nworkers < ntiles) prefetch(next + nworkers);
        if constexpr (PML) {
          // eq. 9 of this tile is done: its sigma buffer takes the next tile's
          if (!mbar_wait_sleep(saddr(mb + B_TZ), ph)) { cfail = true; break; }
          if (next < ntiles) {
            sig_in(next);
            pend_s = it + 1;
          }
        }
        if (!mbar_wait_sleep(saddr(mb + B_OUT), ph)) { cfail = true; break; }
        {  // results are staged in place of the inputs: write them back
          const Tile t = tile_at(tile);
          const uint32_t n = t.ne * 6 * Np * 4;
          const uint32_t eb = ebuf(sl, it), lb = lbuf(sl);
          stage_out(staged(eb + PL::oEQ, P.qin + t.oq), P.qout + t.oq, n);
          stage_out(staged(lb + PL::oLR, P.resq + t.oq), P.resq + t.oq, n);
          if constexpr (PML) {
            stage_out(staged(eb + PL::oEP, P.p + t.op), P.p + t.op, n);
            stage_out(staged(lb + PL::oLRP, P.resp + t.op), P.resp + t.op, n);
          }
          bulk_commit();
          bulk_wait_read();   // staging free for the next tiles
        }
        if (next < ntiles) {
          late_in(next);
          pend_l = it + 1;
          if (EB == 1) {
            early_in(next, it + 1);
            pend_e[0] = it + 1;
          }
        }
      }
      // the staging copies in flight land before the memory is released
      for (int b2 = 0; b2 < 2; ++b2)
        if (pend_e[b2] >= 0 && !mbar_wait_sleep(saddr(mb + B_E0 + b2), eparity(pend_e[b2])))
          cfail = true;
      if (pend_l >= 0 && !mbar_wait_sleep(saddr(mb + B_LATE), pend_l & 1)) cfail = true;
      if (PML && pend_s >= 0 && !mbar_wait_sleep(saddr(mb + B_SIG), pend_s & 1)) cfail = true;
      bulk_wait_all();
      if (cfail) atomicExch(P.err, 1);
    }
    __syncwarp();
  } else if (epilogue_slot<SLOTS, PL::EW>(warp) >= 0) {
    if constexpr (PL::SPLIT) asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(PL::REG_E));
    // ================================================= epilogue warps
    const int sl = epilogue_slot<SLOTS, PL::EW>(warp);
    const int qd = warp & 3, h = warp >> 2;   // quadrant, split
    const uint32_t sA = PL::oA + sl * PL::ASLOT;
    uint64_t* mb = mbar + 12 * sl;
    const int row = 32 * (qd - 2 * sl) + lane;         // row within the slot's tile
    const int e = row >> 3, c = row & 7;
    // this warp's lane quadrant and the slot's columns
    const uint32_t tl = tmem + ((uint32_t)(32 * qd) << 16) + sl * PL::CSTR;
    // curl exchange partners among the six live lanes of an element (pad
    // lanes read themselves): round 1 reads derivative (src + 2) % 3 of lane
    // src1, round 2 derivative (src + 1) % 3 of lane src2; the lane tables
    // (5,3,4,2,0,1) and (4,5,3,1,2,0) packed one nibble per component
    const int base = lane & ~7;
    const int s1 = base + (c < 6 ? (0x102435 >> (4 * c)) & 15 : c);
    const int s2 = base + (c < 6 ? (0x021354 >> (4 * c)) & 15 : c);
    const int send1 = (c + 2) % 3, send2 = (c + 1) % 3;
    const int i0 = h * PL::NS, i1 = min(Np, i0 + PL::NS);   // nodes of this split
    int it = 0;
    for (int tile = blockIdx.x * SLOTS + sl; tile < ntiles && !failed; tile += nworkers, ++it) {
      const uint32_t ph = it & 1;
      const Tile t = tile_at(tile);
      const int ne = t.ne;
      const bool live = c < 6 && e < ne;
      const uint32_t eb = ebuf(sl, it), lb = lbuf(sl);
      if (!mbar_wait_sleep(saddr(mb + B_E0 + (EB == 2 ? (it & 1) : 0)), eparity(it))) {
        failed = true;
        break;
      }
      float* SQ = reinterpret_cast<float*>(staged(eb + PL::oEQ, P.qin + t.oq));
      float* SP = PML ? reinterpret_cast<float*>(staged(eb + PL::oEP, P.p + t.op)) : nullptr;
      // ---- A operands: this thread's row (e, c), its half of the K chunks
      // (every value loaded before any is stored: the staging and operand
      // buffers are all shared memory, so stores would otherwise order the
      // later loads behind them)
      {
        constexpr int NCH = NpK / CW;
        constexpr int H0 = (NCH + PL::S - 1) / PL::S;   // chunks per split
        const int k0 = h * H0, nch = max(0, min(H0, NCH - k0));
        const float* fq = SQ + (e * 6 + c) * Np;
        const float* fp = PML ? SP + (e * 6 + c) * Np : nullptr;
        float x[H0 * CW], y[PML ? H0 * CW : 1];
#pragma unroll
        for (int u = 0; u < H0 * CW; ++u) {
          const int k = k0 * CW + u;
          const bool ok = live && u < nch * CW && k < Np;
          x[u] = ok ? fq[k] : 0.f;
          if constexpr (PML) y[u] = ok ? fp[k] : 0.f;
        }
#pragma unroll
        for (int kc = 0; kc < H0; ++kc) {
          if (kc >= nch) break;
          const uint32_t o = cofs<BF>(row, (k0 + kc) * CW, PL::SBF, 128);
          const float* xx = x + kc * CW;
          if constexpr (BF) {
            uint32_t w[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const __nv_bfloat162 v2 = __floats2bfloat162_rn(xx[2 * u], xx[2 * u + 1]);
              w[u] = *reinterpret_cast<const uint32_t*>(&v2);
            }
            *reinterpret_cast<uint4*>(smem + sA + PL::oAF + o) = make_uint4(w[0], w[1], w[2], w[3]);
            if constexpr (PML) {
              const float* yy = y + kc * CW;
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const __nv_bfloat162 v2 = __floats2bfloat162_rn(yy[2 * u], yy[2 * u + 1]);
                w[u] = *reinterpret_cast<const uint32_t*>(&v2);
              }
              *reinterpret_cast<uint4*>(smem + sA + PL::oAP + o) =
                  make_uint4(w[0], w[1], w[2], w[3]);
            }
          } else {
            *reinterpret_cast<float4*>(smem + sA + PL::oAF + o) =
                make_float4(to_tf32_int(xx[0]), to_tf32_int(xx[1]), to_tf32_int(xx[2]), to_tf32_int(xx[3]));
            if constexpr (PML) {
              const float* yy = y + kc * CW;
              *reinterpret_cast<float4*>(smem + sA + PL::oAP + o) =
                  make_float4(to_tf32_int(yy[0]), to_tf32_int(yy[1]), to_tf32_int(yy[2]), to_tf32_int(yy[3]));
            }
          }
        }
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(saddr(mb + B_FP));
      // this element's metric (r_x .. t_z) and 1/eps, 1/mu
      float g[9], ie, im;
      {
        const float* met =
            reinterpret_cast<const float*>(staged(eb + PL::oEMET, P.geof + t.eg0 * 9));
        const float* mat = reinterpret_cast<const float*>(staged(eb + PL::oEMAT, P.mat + t.eg0 * 3));
        const int ee = e < ne ? e : 0;
#pragma unroll
        for (int j = 0; j < 9; ++j) g[j] = met[ee * 9 + j];
        ie = mat[ee * 3 + 0];
        im = mat[ee * 3 + 1];
      }
      if constexpr (PML) {
        // ---- eq. 9 at this half's quadrature points -> T and Z rows
        if (!mbar_wait_sleep(saddr(mb + B_V), ph)) { failed = true; break; }
        fence_after();
        if (!mbar_wait_sleep(saddr(mb + B_SIG), ph)) { failed = true; break; }
        const float* sg = reinterpret_cast<const float*>(
            staged(lb + PL::oLSG, P.sig + (t.eg0 - P.K0) * 3 * NqP));
        const float ie0 = 1.f / (float)P.eps0;
        const int u = c % 3;
        const int ee = e < ne ? e : 0;
        // the lanes of one element need the axes in the orders (u, v, w) =
        // (0,1,2), (1,2,0), (2,0,1).  Where rows 0 and 2 (2 NqP floats
        // apart) fall on the same banks, the TF32 kernel has every lane read
        // the rows in axis order (one address per element and load) and
        // permute them in registers; otherwise, and in the BF16 kernel
        // (measured faster there), each lane reads its own order.
        constexpr bool ordered = !BF && (2 * NqP) % 32 == 0;
        const float* s0_p = sg + (ee * 3) * NqP;
        const float* su_p = sg + (ee * 3 + u) * NqP;
        const float* sv_p = sg + (ee * 3 + (u == 2 ? 0 : u + 1)) * NqP;
        const float* sw_p = sg + (ee * 3 + (u == 0 ? 2 : u - 1)) * NqP;
        const int q0 = h * PL::QS, q1 = min(NqK, q0 + PL::QS);
        constexpr int QB = 8;    // points per batch of tensor-memory loads
        for (int qq = q0; qq < q1; qq += QB) {
          // V_q of the F row and of the P row at points qq .. qq + 15, one wait
          uint32_t rv[2 * QB];
          tld_cols_nw<QB>(tl + PL::cVF + qq, rv);
          tld_cols_nw<QB>(tl + PL::cVP + qq, rv + QB);
          // sigma of the three axes at points qq .. qq + 15 (16-byte aligned;
          // entries past the capacity hold zeros, and the rule's padding
          // points carry zero weight in P_q), loaded before any store and
          // while the tensor-memory loads are in flight
          float4 sgu[QB / 4], sgv[QB / 4], sgw[QB / 4];
#pragma unroll
          for (int j4 = 0; j4 < QB / 4; ++j4) {
            const int qb = qq + 4 * j4;
            sgu[j4] = sgv[j4] = sgw[j4] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (qb < NqP && qb < q1) {
              if constexpr (!ordered) {
                sgu[j4] = *reinterpret_cast<const float4*>(su_p + qb);
                sgv[j4] = *reinterpret_cast<const float4*>(sv_p + qb);
                sgw[j4] = *reinterpret_cast<const float4*>(sw_p + qb);
              } else {
                const float4 a0 = *reinterpret_cast<const float4*>(s0_p + qb);
                const float4 a1 = *reinterpret_cast<const float4*>(s0_p + NqP + qb);
                const float4 a2 = *reinterpret_cast<const float4*>(s0_p + 2 * NqP + qb);
                sgu[j4] = u == 0 ? a0 : (u == 1 ? a1 : a2);
                sgv[j4] = u == 0 ? a1 : (u == 1 ? a2 : a0);
                sgw[j4] = u == 0 ? a2 : (u == 1 ? a0 : a1);
              }
            }
          }
          tmem_wait_ld();
          float tz[2][QB];
#pragma unroll
          for (int j4 = 0; j4 < QB / 4; ++j4) {
            const float sa[4] = {sgu[j4].x, sgu[j4].y, sgu[j4].z, sgu[j4].w};
            const float sb4[4] = {sgv[j4].x, sgv[j4].y, sgv[j4].z, sgv[j4].w};
            const float sc4[4] = {sgw[j4].x, sgw[j4].y, sgw[j4].z, sgw[j4].w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int jj = 4 * j4 + j;
              const float vf = __uint_as_float(rv[jj]), vp = __uint_as_float(rv[QB + jj]);
              const float su = sa[j] * ie0, sv = sb4[j] * ie0, sw = sc4[j] * ie0;
              // eq. 9 with kappa = 1 in terms of s = sigma / eps0:
              // b = sv + sw - su, c = sv sw - b su, d = su
              const float bc = sv + sw - su;
              const float cc = sv * sw - bc * su;
              const bool ok = live && qq + jj < Nq;
              tz[0][jj] = ok ? bc * vf + cc * vp : 0.f;
              tz[1][jj] = ok ? vf - su * vp : 0.f;
            }
          }
          // K chunks of CW points (4 TF32 / 8 BF16) of the T and Z rows
#pragma unroll
          for (int cj = 0; cj < QB / CW; ++cj) {
            const int k = qq + cj * CW;
            if (k >= q1) break;
            const uint32_t o = cofs<BF>(row, k, PL::SBT, 128);
            const float* t0p = tz[0] + cj * CW;
            const float* z0p = tz[1] + cj * CW;
            if constexpr (BF) {
              uint32_t w0[4], w1[4];
#pragma unroll
              for (int u2 = 0; u2 < 4; ++u2) {
                const __nv_bfloat162 a2 = __floats2bfloat162_rn(t0p[2 * u2], t0p[2 * u2 + 1]);
                const __nv_bfloat162 b2 = __floats2bfloat162_rn(z0p[2 * u2], z0p[2 * u2 + 1]);
                w0[u2] = *reinterpret_cast<const uint32_t*>(&a2);
                w1[u2] = *reinterpret_cast<const uint32_t*>(&b2);
              }
              *reinterpret_cast<uint4*>(smem + sA + PL::oAF + o) =
                  make_uint4(w0[0], w0[1], w0[2], w0[3]);
              *reinterpret_cast<uint4*>(smem + sA + PL::oAP + o) =
                  make_uint4(w1[0], w1[1], w1[2], w1[3]);
            } else {
              *reinterpret_cast<float4*>(smem + sA + PL::oAF + o) = make_float4(
                  to_tf32_int(t0p[0]), to_tf32_int(t0p[1]), to_tf32_int(t0p[2]),
                  to_tf32_int(t0p[3]));
              *reinterpret_cast<float4*>(smem + sA + PL::oAP + o) = make_float4(
                  to_tf32_int(z0p[0]), to_tf32_int(z0p[1]), to_tf32_int(z0p[2]),
                  to_tf32_int(z0p[3]));
            }
          }
        }
        fence_async_smem();
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(saddr(mb + B_TZ));
      }
      // ---- curl with the LIFT term: right-hand side of E, H at this half's
      // nodes, kept in registers until the update
      if (!mbar_wait_sleep(saddr(mb + B_L), ph)) { failed = true; break; }
      fence_after();
      constexpr int NHC = PL::NS;
      float rhs[NHC];
      const int eg = (int)t.eg0 + (e < ne ? e : 0);
      // one batch of nb nodes from node offset ic: d/dr, d/ds, d/dt, LIFT
      auto curl_batch = [&](auto nbc, int ic) {
        constexpr int nb = decltype(nbc)::value;
        const int i = i0 + ic;
        uint32_t r[4 * nb];
        tld_cols_nw<nb>(tl + PL::cD + i, r);
        tld_cols_nw<nb>(tl + PL::cD + NpA + i, r + nb);
        tld_cols_nw<nb>(tl + PL::cD + 2 * NpA + i, r + 2 * nb);
        tld_cols_nw<nb>(tl + PL::cL + i, r + 3 * nb);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < nb; ++j) {
          const float dr = __uint_as_float(r[j]), ds = __uint_as_float(r[nb + j]);
          const float dt = __uint_as_float(r[2 * nb + j]), lf = __uint_as_float(r[3 * nb + j]);
          const float dx = g[0] * dr + g[3] * ds + g[6] * dt;
          const float dy = g[1] * dr + g[4] * ds + g[7] * dt;
          const float dz = g[2] * dr + g[5] * ds + g[8] * dt;
          const float o1 = send1 == 0 ? dx : (send1 == 1 ? dy : dz);
          const float o2 = send2 == 0 ? dx : (send2 == 1 ? dy : dz);
          const float a1 = __shfl_sync(0xffffffffu, o1, s1);
          const float a2 = __shfl_sync(0xffffffffu, o2, s2);
          const float cr = a1 - a2 + lf;   // (curl of the partner field) + LIFT term
          rhs[ic + j] = c < 3 ? ie * cr : -im * cr;
        }
      };
      constexpr int CB = NHC < 12 ? NHC : 12;   // nodes per batch of loads
#pragma unroll
      for (int ic = 0; ic + CB <= NHC; ic += CB) curl_batch(std::integral_constant<int, CB>{}, ic);
      if constexpr (NHC % CB != 0)
        curl_batch(std::integral_constant<int, NHC % CB>{}, NHC - NHC % CB);
      // dipole sources of this element (E rows): -J(t) dir M_k^-1 l(r_s)
      if (live && c < 3) {
        for (int s = 0; s < P.nsrc; ++s) {
          const int sb = s < kSrcCache ? srcc[2 * s] : P.src[s].batch;
          const int se = s < kSrcCache ? srcc[2 * s + 1] : P.src[s].elem;
          if (sb != t.b || se != eg) continue;
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
      // the P_q outputs (s for E, H rows; the right-hand side for P rows)
      uint32_t sz[2 * NHC];
      if constexpr (PML) {
        if (!mbar_wait_sleep(saddr(mb + B_PQ), ph)) { failed = true; break; }
        fence_after();
        tld_cols_nw<NHC>(tl + PL::cVF + i0, sz);
        tld_cols_nw<NHC>(tl + PL::cVP + i0, sz + NHC);
        tmem_wait_ld();
      }
      if (!mbar_wait_sleep(saddr(mb + B_LATE), ph)) { failed = true; break; }
      float* SR = reinterpret_cast<float*>(staged(lb + PL::oLR, P.resq + t.oq));
      float* SRP = PML ? reinterpret_cast<float*>(staged(lb + PL::oLRP, P.resp + t.op)) : nullptr;
      // ---- Runge-Kutta update of this half's nodes, in place in the staging:
      // batches of UB nodes, every value of a batch loaded before any store
      if (live) {
        constexpr int UB = 5;
        float* sr = SR + (e * 6 + c) * Np;
        float* sq = SQ + (e * 6 + c) * Np;
        float* srp = PML ? SRP + (e * 6 + c) * Np : nullptr;
        float* spp = PML ? SP + (e * 6 + c) * Np : nullptr;
#pragma unroll
        for (int j0 = 0; j0 < NHC; j0 += UB) {
          float r_[UB], q_[UB], rp_[UB], p_[UB];
#pragma unroll
          for (int j = 0; j < UB; ++j) {
            const int ii = i0 + j0 + j;
            if (j0 + j < NHC && ii < i1) {
              r_[j] = sr[ii];
              q_[j] = sq[ii];
              if constexpr (PML) {
                rp_[j] = srp[ii];
                p_[j] = spp[ii];
              }
            }
          }
#pragma unroll
          for (int j = 0; j < UB; ++j) {
            const int ii = i0 + j0 + j;
            if (j0 + j >= NHC || ii >= i1) break;
            const float s_ = PML ? __uint_as_float(sz[j0 + j]) : 0.f;
            const float rr = rka * r_[j] + rdt * (rhs[j0 + j] - s_);
            sr[ii] = rr;
            sq[ii] = q_[j] + rkb * rr;
            if constexpr (PML) {
              const float rp = rka * rp_[j] + rdt * __uint_as_float(sz[NHC + j0 + j]);
              srp[ii] = rp;
              spp[ii] = p_[j] + rkb * rp;
            }
          }
        }
      }
      fence_async_smem();   // the bulk copies read these values
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(saddr(mb + B_OUT));
    }
    if (failed && lane == 0) atomicExch(P.err, 1);
  } else {
    if constexpr (PL::SPLIT) asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(PL::REG_F));
    // ================================================= flux warps
    int fidx = 0;
    const int sl = flux_slot<SLOTS, PL::EW>(warp, fidx);
    const uint32_t sA = PL::oA + sl * PL::ASLOT;
    uint64_t* mb = mbar + 12 * sl;
    const int ft = fidx * 32 + lane;   // flux thread of the slot
    constexpr int NFT = 32 * PL::FLUXW;
    constexpr int FT = (T * NF + NFT - 1) / NFT;    // tasks per thread
    // neighbour traces of a tile (global memory), loaded one tile ahead; the
    // tile's neighbour and code tables come from its early buffer
    float Ep[FT][3], Hp[FT][3], ZPv[FT];
    // (with two early buffers the tile's neighbour tables come from its
    // early buffer, iteration itn: false if that wait gave up)
    auto load_nbr = [&](int tile, int itn) -> bool {
      const Tile t = tile_at(tile);
      const float* qin = P.qin + (int64_t)t.b * P.strideQ;
      const int* nbs = P.nbr + t.eg0 * 4;
      const unsigned char* cds = P.code + t.eg0 * 4;
      if constexpr (EB == 2) {
        if (!mbar_wait_sleep(saddr(mb + B_E0 + (itn & 1)), eparity(itn))) return false;
        nbs = reinterpret_cast<const int*>(staged(ebuf(sl, itn) + PL::oENB, nbs));
        cds = staged(ebuf(sl, itn) + PL::oECD, cds);
      }
#pragma unroll
      for (int u = 0; u < FT; ++u) {
        const int task = ft + u * NFT;
        ZPv[u] = -1.f;
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) { Ep[u][cc] = 0.f; Hp[u][cc] = 0.f; }
        if (task < t.ne * NF) {
          const int e = task / NF, fm = task - e * NF, f = fm / Nfp, m = fm - f * Nfp;
          const int nb = nbs[e * 4 + f];
          if (nb >= 0) {
            const int code = cds[e * 4 + f];
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
      return true;
    };
    const int first = blockIdx.x * SLOTS + sl;
    if (first < ntiles && !load_nbr(first, 0)) failed = true;
    int it = 0;
    for (int tile = first; tile < ntiles && !failed; tile += nworkers, ++it) {
      const uint32_t ph = it & 1;
      const Tile t = tile_at(tile);
      const uint32_t eb = ebuf(sl, it);
      if (!mbar_wait_sleep(saddr(mb + B_E0 + (EB == 2 ? (it & 1) : 0)), eparity(it))) {
        failed = true;
        break;
      }
      // the previous tile's LIFT product has read the flux operand
      if (it > 0 && !mbar_wait_sleep(saddr(mb + B_L), ph ^ 1)) { failed = true; break; }
      const float* SQ = reinterpret_cast<const float*>(staged(eb + PL::oEQ, P.qin + t.oq));
      const float* fn_s = reinterpret_cast<const float*>(staged(eb + PL::oEFN, P.fnrm + t.eg0 * 16));
      const float* mat_s = reinterpret_cast<const float*>(staged(eb + PL::oEMAT, P.mat + t.eg0 * 3));
      const float al = (float)P.alpha;
#pragma unroll
      for (int u = 0; u < FT; ++u) {
        const int task = ft + u * NFT;
        if (task >= t.ne * NF) continue;
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
        const uint32_t o = cofs<BF>(8 * e, fm, PL::SBLA, PL::LBA);
#pragma unroll
        for (int cc = 0; cc < 6; ++cc) {
          unsigned char* dst = smem + sA + PL::oAL + o + 16 * cc;
          if constexpr (BF) *reinterpret_cast<__nv_bfloat16*>(dst) = __float2bfloat16_rn(fo[cc]);
          else *reinterpret_cast<float*>(dst) = to_tf32_int(fo[cc]);
        }
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(saddr(mb + B_FLUX));
      // the next tile's neighbour traces load while this tile's epilogue runs
      if (tile + nworkers < ntiles && !load_nbr(tile + nworkers, it + 1)) {
        failed = true;
        break;
      }
    }
    if (failed && lane == 0) atomicExch(P.err, 1);
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) tmem_dealloc(tmem, PL::TMEM_COLS);
}

template <int N, bool PML, bool BF>
cudaError_t rows_configure() {
  using PL = RPlan<N, PML, BF>;
  // setmaxnreg.inc waits until the block's launch allocation covers the
  // split: refuse a build whose compiled register count would leave it short
  if constexpr (PL::SPLIT) {
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, tc_rows_kernel<N, PML, BF>);
    if (e != cudaSuccess) return e;
    if ((long)fa.numRegs * PL::THREADS <
        32L * (PL::EW * PL::REG_E + 4 * PL::REG_F + 4 * PL::REG_C))
      return cudaErrorInvalidConfiguration;
  }
  return cudaFuncSetAttribute(tc_rows_kernel<N, PML, BF>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)PL::bytes);
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
  const int grid = (int)std::min<long long>((tiles + PL::SLOTS - 1) / PL::SLOTS, (long long)sms);
  tc_rows_kernel<N, PML, BF><<<grid, PL::THREADS, PL::bytes, s>>>(Q);
  return cudaGetLastError();
}

}  // namespace tc

template <bool BF>
cudaError_t configure_rows(int N) {
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
  return bf16 ? configure_rows<true>(N) : configure_rows<false>(N);
}

template <bool BF>
cudaError_t launch_rows(int N, const StageParams<float>& P, int nb, cudaStream_t s) {
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
  // the bulk copies move whole 16-byte covers of each block: the arrays must
  // start on 16-byte boundaries (cudaMalloc gives 256)
  const uintptr_t a =
      reinterpret_cast<uintptr_t>(P.qin) | reinterpret_cast<uintptr_t>(P.qout) |
      reinterpret_cast<uintptr_t>(P.resq) | reinterpret_cast<uintptr_t>(P.p) |
      reinterpret_cast<uintptr_t>(P.resp) | reinterpret_cast<uintptr_t>(P.sig) |
      reinterpret_cast<uintptr_t>(P.fnrm) | reinterpret_cast<uintptr_t>(P.geof) |
      reinterpret_cast<uintptr_t>(P.mat);
  if (a & 15) return cudaErrorMisalignedAddress;
  return bf16 ? launch_rows<true>(N, P, nb, s) : launch_rows<false>(N, P, nb, s);
}

}  // namespace wadg
