// Tensor-core stage kernels for sm_103a (tcgen05, TF32 or BF16 operands, FP32
// accumulation in tensor memory, FP32 field state).
//
// Every reference-element contraction of the stage is one matrix product
//     D[row][(e,c)] = sum_k A[row][k] * B[(e,c)][k]
// with the operator as A (rows = output node or quadrature point, which
// become TMEM lanes) and the tile's field data as B (one row per
// (element, component) pair, K-major), so each thread of the epilogue owns one
// node / quadrature point of every element of the tile:
//   volume  : A = Dr, Ds, Dt  (Np x Np)   B = E,H           -> d/dr, d/ds, d/dt
//   LIFT    : A = LIFT (Np x 4Nfp)        B = scaled flux   -> surface term
//   PML     : A = V_q (Nq x Np)           B = E,H,P^E,P^H   -> values at x_q
//             A = P_q (Np x Nq)           B = (t, z) at x_q -> s, rhs of P
// (eqs. 16, 17, 20, 21, 26-29).  The upwind flux, the metric chain rule,
// eq. 9 at the quadrature points and the Runge-Kutta update run on the CUDA
// cores between the products.  Operand tiles use the K-major canonical
// layout without swizzle: 8-row x 16-byte core matrices, K-adjacent core
// matrices 128 B apart (LBO), 8-row groups SBO apart.  M = 128 always;
// operators with fewer rows are stored with their real rows only and the
// rows the instruction reads beyond them fall on later shared-memory buffers
// (their lanes are never read back).
//
// Waits on the MMA-completion mbarrier are bounded; on timeout the kernel
// records an error and stops after releasing its tensor memory.
#include "kernels.cuh"
#include "tc_ptx.cuh"

#include <algorithm>
#include <cstdint>

namespace wadg {
namespace tc {

// Shared-memory plan of one tile (all offsets in bytes).  QC: quadrature
// class of the volume rule (quad_capacity).
template <int N, bool PML, bool BF = false, int QC = 0>
struct Plan {
  using O = OpT<BF>;
  static constexpr int Np = (N + 1) * (N + 2) * (N + 3) / 6;
  static constexpr int Nfp = (N + 1) * (N + 2) / 2;
  static constexpr int NF = 4 * Nfp;
  static constexpr int Nq = quad_capacity(N, QC);
  __host__ __device__ static constexpr int rupK(int x) { return (x + O::KS - 1) / O::KS * O::KS; }
  static constexpr int NpK = rupK(Np), NFK = rupK(NF), NqK = rupK(Nq);
  // elements per tile: 8; 4 for BF16 PML tiles, whose smaller operands then
  // let two blocks share an SM (N <= 4) or fit at all (N = 5), and for TF32
  // PML tiles at N = 5 (compact rule only)
  static constexpr bool PAIR = PML && BF && N <= 4;
  static constexpr int T = PML && (BF || N == 5) ? 4 : 8;
  // one block per SM with 16 compute warps (TF32 PML; every N = 5 tile)
  static constexpr bool ONE = PML ? !PAIR : N == 5;
  static constexpr int NV = rup16(6 * T);            // columns of E,H products
  static constexpr int NQ = rup16(12 * T);           // columns of 12-component products
  static constexpr int G_p = NpK / 8;                // 8-row groups of an Np-row operator
  static constexpr uint32_t LA = 128, LB = 144;      // K strides of operator / field tiles
  static constexpr uint32_t SBO_V = (NpK / O::CW) * LA;  // operators, K = Np
  static constexpr uint32_t SBO_L = (NFK / O::CW) * LA;  // K = 4 Nfp
  static constexpr uint32_t SBO_Q = (NqK / O::CW) * LA;  // K = Nq
  static constexpr uint32_t SBB_V = (NpK / O::CW) * LB;  // field tiles
  static constexpr uint32_t SBB_L = (NFK / O::CW) * LB;
  static constexpr uint32_t SBB_Q = (NqK / O::CW) * LB;
  __host__ __device__ static constexpr uint32_t ofs(int r, int k, uint32_t sbo, uint32_t lbo) {
    return cofs<BF>(r, k, sbo, lbo);
  }
  // A operands
  static constexpr uint32_t oPq = 0;
  static constexpr uint32_t oL = PML ? oPq + G_p * SBO_Q : 0;
  // Dr, Ds, Dt stacked as one operator of 3 Np rows (row d Np + i), read as
  // VT products of up to 128 rows: DPT derivatives per product (N <= 4: all
  // three in one; N = 5: [Dr; Ds], then Dt)
  static constexpr int DPT = (128 / Np) < 3 ? (128 / Np) : 3;
  static constexpr int VT = (3 + DPT - 1) / DPT;
  static constexpr int RV = rup8(3 * Np);
  static constexpr uint32_t oVol = oL + G_p * SBO_L;
  static constexpr uint32_t oVq = oVol + (RV / 8) * SBO_V;
  // V_q read as VQT products of 128 rows (quadrature points q and q + 128);
  // the rows an instruction reads past the operator's own fall on the
  // buffers that follow it
  static constexpr int VQT = (Nq + 127) / 128;
  // B operands
  static constexpr uint32_t oBF = PML ? oVq + (rup8(Nq) / 8) * SBO_V : oVq;
  static constexpr int ROWS_F = PML ? NQ : NV;        // E,H (+ P) rows
  static constexpr uint32_t oBFL = oBF + (ROWS_F / 8) * SBB_V;
  static constexpr uint32_t oBTZ = oBFL + (NV / 8) * SBB_L;
  // the (t, z) operand buffer later holds the P_q columns copied out of
  // TMEM ([T][12][Np] floats), which can be the larger of the two
  static constexpr uint32_t BTZ_BYTES = (NQ / 8) * SBB_Q;
  static constexpr uint32_t DP_BYTES = T * 12 * Np * 4;
  static constexpr uint32_t oRS =
      PML ? oBTZ + (BTZ_BYTES > DP_BYTES ? BTZ_BYTES : DP_BYTES) : oBTZ;
  static constexpr int NpP = (Np + 3) & ~3;
  static constexpr uint32_t oGeo = oRS + (PML ? T * 6 * NpP * 4 : 0);
  static constexpr int TS = T * 6 * Np;               // floats of one staged field block
  // a staged block is the 16-byte-aligned cover of the element block: up to
  // 8 bytes more at each end
  static constexpr uint32_t TSB = ((TS * 4 + 15) & ~15) + 16;
  // a staging set: q, res (+ P, res of P), then the tile's geometry blocks as
  // stored in global memory (covers again): unit normal and Fscale [T][4][4]
  // floats, metric [T][9] doubles, 1/eps, 1/mu, Z [T][3] floats
  static constexpr uint32_t GFN = ((T * 64 + 15) & ~15) + 16;
  static constexpr uint32_t GMET = ((T * 72 + 15) & ~15) + 16;
  static constexpr uint32_t GMAT = ((T * 12 + 15) & ~15) + 16;
  static constexpr uint32_t oSFN = (PML ? 4 : 2) * TSB;   // offsets within a set
  static constexpr uint32_t oSMET = oSFN + GFN;
  static constexpr uint32_t oSMAT = oSMET + GMET;
  static constexpr uint32_t SET = oSMAT + GMAT;
  // the current tile's metric (9) and 1/eps, 1/mu in float [T][12]
  static constexpr uint32_t oST = oGeo + ((T * 12 * 4 + 15) & ~15u);  // two staging sets
  static constexpr uint32_t oMisc = oST + 2 * SET;
  // misc: 10 mbarriers | TMEM slot | flags | tile source list (64) | cached
  // (batch, element) of the first 64 sources | face tables (Fmask, fperm)
  static constexpr uint32_t oTabs = 896;
  static constexpr uint32_t MISC_BYTES = (oTabs + 100 * Nfp + 15) & ~15u;
  // epilogue scratch: the node rows of the products copied out of TMEM so that
  // every warp can share the per-node work.  PML: the volume/LIFT columns go
  // to the field-operand buffers (free once the first products are done), the
  // P_q columns to the (t, z) buffer (free once P_q is done).
  // [T][6][4][Np] (component, d/dr d/ds d/dt LIFT, node) with an element
  // stride DVE = Np (mod 32): a warp's stores (consecutive derivative-node
  // pairs of one element) and its loads (consecutive element-node pairs) both
  // fall on 32 distinct banks
  static constexpr int DVE = 24 * Np + ((Np - 24 * Np) % 32 + 32) % 32;
  static constexpr uint32_t DV_BYTES = T * DVE * 4;
  // (BF16 operand buffers are too small for the volume/LIFT dump: it gets its
  // own region)
  static constexpr bool DV_ALIAS = PML && !BF;
  static constexpr uint32_t oDV = DV_ALIAS ? oBF : oMisc + MISC_BYTES;
  static constexpr uint32_t oDP = oBTZ;
  static_assert(!DV_ALIAS || oDV + DV_BYTES <= oBTZ, "volume/LIFT dump");
  static_assert(!PML || oDP + DP_BYTES <= oRS, "P_q dump");
  static constexpr uint32_t bytes_used = DV_ALIAS ? oMisc + MISC_BYTES : oDV + DV_BYTES;
  // residency follows the tensor-memory budget of 512 columns per SM: one
  // TF32 PML block (512 columns) per SM, enforced by the shared-memory request
  // so that no block waits in tcgen05.alloc; BF16 PML blocks (256 columns)
  // and non-PML blocks (128 columns) two per SM (shared memory, registers)
  static constexpr uint32_t min_bytes = ONE ? 116 * 1024 : 100 * 1024;
  static constexpr uint32_t bytes = bytes_used < min_bytes ? min_bytes : bytes_used;
  // TMEM column bases: derivative products (lanes d Np + i of product v at
  // cV + v NV), LIFT, V_q products (cVq + t NQ), P_q
  static constexpr uint32_t cV = 0, cL = VT * NV;
  static constexpr uint32_t cVq = cL + NV, cPq = cVq + VQT * NQ;
  static constexpr uint32_t COLS = PML ? cPq + NQ : cL + NV;
  static constexpr uint32_t TMEM_COLS = COLS <= 128 ? 128 : (COLS <= 256 ? 256 : 512);
  static_assert(COLS <= 512, "TMEM columns");
  static_assert(!PAIR || (bytes <= 113 * 1024 && TMEM_COLS <= 256), "two BF16 PML blocks per SM");
  static_assert(ONE || TMEM_COLS <= 256, "two blocks per SM");
  static_assert((DPT * Np) % 8 == 0 || VT == 1, "second derivative product starts on a row group");
  static_assert(VT <= 2 && VQT <= 2, "at most two products per operator");
  static_assert(Np <= 64, "node rows");
  // every A operand read (128 rows from its start) stays inside the block
  static_assert(oPq + 16 * SBO_Q <= bytes || !PML, "P_q span");
  static_assert(oL + 16 * SBO_L <= bytes, "LIFT span");
  static_assert(oVol + ((VT - 1) * DPT * Np / 8 + 16) * SBO_V <= bytes, "volume operator span");
  static_assert(!PML || oVq + 16 * VQT * SBO_V <= bytes, "V_q span");
  static_assert(VQT == 1 || Nq % 8 == 0, "second V_q product starts on a row group");
  static_assert(bytes <= 227 * 1024, "shared memory");
};

// Warp roles.  The compute warps (16 in a one-per-SM block: TF32 PML and the
// N = 5 BF16 blocks; 8 in a block that shares its SM with another) stage the
// tile, build the operands, compute the flux and run the epilogues; they
// synchronise among themselves on a named barrier.  An issuing warpgroup
// follows them: lane 0 of its first warp waits for "operand ready" mbarriers
// the compute warps arrive on and commits each product to a "product done"
// mbarrier, so that issuing the products (about a hundred cycles per
// instruction for the issuing thread) stays off the compute warps' path.  The
// issuing warpgroup keeps 24 registers per thread and hands the rest of its
// launch allocation to the compute warps (setmaxnreg), which removes their
// spills (the launch holds every thread to the share of 5 or 6 warps per
// scheduler).
template <int N, bool PML, bool BF, int QC = 0>
struct TcWarps {
  static constexpr bool ONE = Plan<N, PML, BF, QC>::ONE;   // one block per SM
  static constexpr int compute = ONE ? 16 : 8;
  static constexpr int issue = 4;
  static constexpr int threads = 32 * (compute + issue);
  // registers per thread at launch, of the issuing warpgroup after it gives
  // its share away, and of the compute warps after they take it (the block's
  // launch allocation covers both: checked against the compiled kernel before
  // the first launch)
  static constexpr int launch_regs = ONE ? 96 : 80;
  static constexpr int issue_regs = 24;
  static constexpr int compute_regs =
      ((threads * launch_regs - 32 * issue * issue_regs) / (32 * compute)) & ~7;
  static_assert(compute_regs >= launch_regs && compute_regs <= 256, "register split");
  static_assert(32 * compute * compute_regs + 32 * issue * issue_regs <= threads * launch_regs,
                "register split within the launch allocation");
};

template <int N, bool PML, bool BF, int QC>
__global__ void __launch_bounds__(TcWarps<N, PML, BF, QC>::threads,
                                  TcWarps<N, PML, BF, QC>::ONE ? 1 : 2)
    tc_stage_kernel(const StageParams<float> P) {
  using PL = Plan<N, PML, BF, QC>;
  using TW = TcWarps<N, PML, BF, QC>;
  constexpr int NW = TW::compute;
  constexpr int kTcThreads = 32 * NW;          // compute threads
  constexpr int kAll = TW::threads;
  constexpr int NGRP = NW / 4;                 // warps sharing a TMEM lane quadrant
  constexpr int Np = PL::Np, Nfp = PL::Nfp, NF = PL::NF, Nq = PL::Nq, T = PL::T;
  constexpr int NpK = PL::NpK, NFK = PL::NFK, NqK = PL::NqK;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool mma_warp = warp >= NW;   // the issuing warpgroup
  const int quad = warp & 3, grp = warp >> 2;   // TMEM lane quadrant, element group
  const uint32_t sbase = saddr(smem);
  float* RS = reinterpret_cast<float*>(smem + PL::oRS);     // [T][6][NpP]
  float* geoM = reinterpret_cast<float*>(smem + PL::oGeo);  // [T][12]: metric | 1/eps, 1/mu
  // mbarriers: products done [0] V_q, [1] volume + LIFT, [2] P_q; operands
  // ready [3] fields, [4] flux, [5] (t, z); [6] final drain of the MMA warp;
  // [7], [8] staging set 0 / 1 landed
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + PL::oMisc);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + PL::oMisc + 80);
  int* flags = reinterpret_cast<int*>(smem + PL::oMisc + 84);   // [0] source count
  int* srcl = reinterpret_cast<int*>(smem + PL::oMisc + 112);
  int* srcc = reinterpret_cast<int*>(smem + PL::oMisc + 368);   // [64][2] batch, element
  constexpr int kSrcCache = 64;
  const float* tops = reinterpret_cast<const float*>(P.tcops);
  // face-node tables, copied to shared memory in the prologue: Fmask [NF],
  // fperm [4][24][Nfp]
  unsigned char* tabs_s = smem + PL::oMisc + PL::oTabs;
  const unsigned char* Fmask = tabs_s;
  const unsigned char* fperm = tabs_s + NF;

  // ---- prologue: zero the operand buffers, stage the operators
  for (uint32_t i = tid; i < PL::oGeo / 16; i += kAll)
    reinterpret_cast<float4*>(smem)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();
  {
    // tcops layout: Dr | Ds | Dt [Np][Np], LIFT [Np][NF], Vq [Nq][Np], Pq [Np][Nq]
    const float* gDr = tops;
    const float* gL = gDr + 3 * Np * Np;
    const float* gVq = gL + Np * NF;
    const float* gPq = gVq + Nq * Np;
    for (int idx = tid; idx < 3 * Np * Np; idx += kAll) {
      const int row = idx / Np, j = idx - row * Np;   // row d Np + i of [Dr; Ds; Dt]
      put_op<BF>(smem + PL::oVol + PL::ofs(row, j, PL::SBO_V, PL::LA), gDr[idx]);
    }
    for (int idx = tid; idx < Np * NF; idx += kAll) {
      const int i = idx / NF, f = idx - i * NF;
      put_op<BF>(smem + PL::oL + PL::ofs(i, f, PL::SBO_L, PL::LA), gL[idx]);
    }
    if (PML) {
      for (int idx = tid; idx < Nq * Np; idx += kAll) {
        const int q = idx / Np, j = idx - q * Np;
        put_op<BF>(smem + PL::oVq + PL::ofs(q, j, PL::SBO_V, PL::LA), gVq[idx]);
      }
      for (int idx = tid; idx < Np * Nq; idx += kAll) {
        const int i = idx / Nq, q = idx - i * Nq;
        put_op<BF>(smem + PL::oPq + PL::ofs(i, q, PL::SBO_Q, PL::LA), gPq[idx]);
      }
    }
  }
  for (int s = tid; s < min(P.nsrc, kSrcCache); s += kAll) {
    srcc[2 * s] = P.src[s].batch;
    srcc[2 * s + 1] = P.src[s].elem;
  }
  for (int i = tid; i < 100 * Nfp; i += kAll) tabs_s[i] = P.tabs[i];
  if (tid == 0) {
    for (int i = 0; i < 9; ++i) mbar_init(saddr(mbar + i), i >= 3 && i <= 5 ? NW : 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(saddr(tmem_slot), PL::TMEM_COLS);
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t lane_base = static_cast<uint32_t>(quad * 32) << 16;
  uint32_t phase[3] = {0, 0, 0};   // parity of each product barrier's next completion
  bool failed = false;
  // bounded wait of every compute thread for product barrier i; false if any
  // thread gave up
  auto wait_bar = [&](int i) -> bool {
    const bool ok = mbar_wait(saddr(mbar + i), phase[i]);
    if (ok) phase[i] ^= 1;
    const bool all = cbar_and(kTcThreads, ok);
    fence_after();
    return all;
  };
  // a compute warp's operand writes are complete: make them visible to the
  // tensor core and count the warp on "operand ready" barrier i
  auto signal_ready = [&](int i) {
    fence_async_smem();
    fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(saddr(mbar + i));
  };

  const double tbase = P.t_dev ? *P.t_dev : P.t;
  const double tst = tbase + P.rk_c * P.dt;
  const float rka = (float)P.rk_a, rkb = (float)P.rk_b, rdt = (float)P.dt;
  const int tiles_per_batch = (P.n_elem + T - 1) / T;
  const int ntiles = tiles_per_batch * P.nb;

  constexpr int FT = (T * NF + kTcThreads - 1) / kTcThreads;   // flux tasks per thread

  // A tile's contiguous field blocks (E,H and its register; P and its
  // register in PML tiles) in global memory, and where each lands in staging
  // set `set`: a block is copied as its 16-byte-aligned cover, so its first
  // value sits (address mod 16) bytes into the buffer.  (The library's
  // buffers end with spare bytes, so a cover never leaves its allocation.)
  constexpr int NBLK = PML ? 4 : 2;
  auto tile_blocks = [&](int tile, const float* (&g)[4]) {
    const int b = tile / tiles_per_batch;
    const int t0 = (tile - b * tiles_per_batch) * T;
    const int64_t oq = (int64_t)b * P.strideQ + (int64_t)(P.e_begin + t0) * 6 * Np;
    const int64_t op = (int64_t)b * P.strideP + (int64_t)(P.e_begin + t0 - P.K0) * 6 * Np;
    g[0] = P.qin + oq;
    g[1] = P.resq + oq;
    g[2] = PML ? P.p + op : nullptr;
    g[3] = PML ? P.resp + op : nullptr;
  };
  auto staged = [&](int set, int a, const float* g) {
    return reinterpret_cast<float*>(smem + PL::oST + set * PL::SET + a * PL::TSB +
                                    (reinterpret_cast<uintptr_t>(g) & 15));
  };
  // the MMA thread issues the copies (tile k of this block into set k & 1,
  // once the compute warps have signalled operands of tile k - 1, i.e. have
  // finished with tile k - 2); they complete on staging barrier 7 + set
  auto stage_tile = [&](int tile, int set) {
    const float* g[4];
    tile_blocks(tile, g);
    const int b = tile / tiles_per_batch;
    const int t0 = tile - b * tiles_per_batch;
    const int ne = min(T, P.n_elem - t0 * T);
    const int eg0 = P.e_begin + t0 * T;
    constexpr int NB = NBLK + 3;
    const unsigned char* src[NB];
    uint32_t bytes[NB], dst[NB];
#pragma unroll
    for (int a = 0; a < NBLK; ++a) {
      src[a] = reinterpret_cast<const unsigned char*>(g[a]);
      bytes[a] = ne * 6 * Np * 4;
      dst[a] = a * PL::TSB;
    }
    src[NBLK] = reinterpret_cast<const unsigned char*>(P.fnrm + (int64_t)eg0 * 16);
    bytes[NBLK] = ne * 64;
    dst[NBLK] = PL::oSFN;
    src[NBLK + 1] = reinterpret_cast<const unsigned char*>(P.geo + (int64_t)eg0 * 9);
    bytes[NBLK + 1] = ne * 72;
    dst[NBLK + 1] = PL::oSMET;
    src[NBLK + 2] = reinterpret_cast<const unsigned char*>(P.mat + (int64_t)eg0 * 3);
    bytes[NBLK + 2] = ne * 12;
    dst[NBLK + 2] = PL::oSMAT;
    uint32_t lo[NB], len[NB], total = 0;
#pragma unroll
    for (int a = 0; a < NB; ++a) {
      lo[a] = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(src[a]) & 15);
      len[a] = (lo[a] + bytes[a] + 15) & ~15u;
      total += len[a];
    }
    const uint32_t bar = saddr(mbar + 7 + set);
    fence_async_smem();   // the buffers' earlier reads come before the copies' writes
    mbar_expect_tx(bar, total);
#pragma unroll
    for (int a = 0; a < NB; ++a)
      bulk_g2s(sbase + PL::oST + set * PL::SET + dst[a], src[a] - lo[a], len[a], bar);
  };
  // a staged geometry block of set `set` (offset `o` within the set) whose
  // global copy starts at g
  auto staged_at = [&](int set, uint32_t o, const void* g) {
    return smem + PL::oST + set * PL::SET + o + (reinterpret_cast<uintptr_t>(g) & 15);
  };

  // per-tile scattered loads (neighbour traces, sigma samples, geometry),
  // issued one tile ahead so their latency overlaps the previous tile's work
  constexpr int NqP = (Nq + 3) & ~3;
  constexpr int EH = (T + NGRP - 1) / NGRP;
  // level 1 (no use of the loaded values): neighbour ids and face codes
  auto load_nbr_idx = [&](int tile, int (&nbv)[FT], int (&codev)[FT]) {
    const int b = tile / tiles_per_batch;
    const int t0 = (tile - b * tiles_per_batch) * T;
    const int ne = min(T, P.n_elem - t0);
    const int eg0 = P.e_begin + t0;
#pragma unroll
    for (int u = 0; u < FT; ++u) {
      const int task = tid + u * kTcThreads;
      nbv[u] = -1;
      codev[u] = 0;
      if (task < ne * NF) {
        const int e = task / NF, f = (task - e * NF) / Nfp;
        nbv[u] = P.nbr[(eg0 + e) * 4 + f];
        codev[u] = P.code[(eg0 + e) * 4 + f];
      }
    }
  };
  // level 2: the neighbour traces themselves (issued once the ids are in)
  auto load_nbr_val = [&](int tile, const int (&nbv)[FT], const int (&codev)[FT],
                          float (&Ep)[FT][3], float (&Hp)[FT][3], float (&ZPv)[FT]) {
    const int b = tile / tiles_per_batch;
    const int t0 = (tile - b * tiles_per_batch) * T;
    const int ne = min(T, P.n_elem - t0);
    const float* qin = P.qin + (int64_t)b * P.strideQ;
#pragma unroll
    for (int u = 0; u < FT; ++u) {
      const int task = tid + u * kTcThreads;
      ZPv[u] = -1.f;   // marks the PEC mirror
#pragma unroll
      for (int c = 0; c < 3; ++c) { Ep[u][c] = 0.f; Hp[u][c] = 0.f; }
      if (task < ne * NF && nbv[u] >= 0) {
        const int fm = task % NF;
        const int f = fm / Nfp, m = fm - f * Nfp;
        // checked builds: an index out of range leaves the PEC mirror in place
        if (!WADG_INDEX_OK(nbv[u] < P.strideQ / (6 * Np) && codev[u] < 24, P.err)) continue;
        const int np2 = fperm[(f * 24 + codev[u]) * Nfp + m];
        if (!WADG_INDEX_OK(np2 < Np, P.err)) continue;
        const float* qn = qin + (int64_t)nbv[u] * 6 * Np + np2;
#pragma unroll
        for (int c = 0; c < 3; ++c) { Ep[u][c] = qn[c * Np]; Hp[u][c] = qn[(3 + c) * Np]; }
        ZPv[u] = P.mat[nbv[u] * 3 + 2];
      }
    }
  };
  constexpr int VQT = PL::VQT;
  auto load_sig = [&](int tile, float (&sgv)[PML ? EH : 1][VQT][3]) {
    if (!PML) return;
    const int b = tile / tiles_per_batch;
    const int t0 = (tile - b * tiles_per_batch) * T;
    const int ne = min(T, P.n_elem - t0);
    const int ep0 = P.e_begin + t0 - P.K0;
#pragma unroll
    for (int k = 0; k < (PML ? EH : 1); ++k) {
      const int e = grp + NGRP * k;
#pragma unroll
      for (int t = 0; t < VQT; ++t) {
        const int q = 128 * t + quad * 32 + lane;
        sgv[k][t][0] = sgv[k][t][1] = sgv[k][t][2] = 0.f;
        if (e < ne && q < Nq) {
          const int64_t sb = (int64_t)(ep0 + e) * 3 * NqP + q;
          sgv[k][t][0] = P.sig[sb];
          sgv[k][t][1] = P.sig[sb + NqP];
          sgv[k][t][2] = P.sig[sb + 2 * NqP];
        }
      }
    }
  };
  static_assert(9 * T <= kTcThreads, "one metric entry per thread");
  if (mma_warp) {
    // ---- issuing warpgroup: lane 0 of its first warp issues every product
    // of every tile of this block.  It first hands registers to the compute
    // warps (warpgroup-uniform).
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(TW::issue_regs));
    if (warp == NW && lane == 0) {
      uint32_t rph[3] = {0, 0, 0};   // parity of the operand-ready barriers 3, 4, 5
      bool issued = false, mfail = false;
      auto wait_ready = [&](int i) -> bool {
        const bool ok = mbar_wait(saddr(mbar + 3 + i), rph[i]);
        rph[i] ^= 1;
        fence_after();
        return ok;
      };
      constexpr uint32_t idV = BF ? idesc_bf16(128, PL::NV) : idesc_tf32(128, PL::NV);
      constexpr uint32_t idQ = BF ? idesc_bf16(128, PL::NQ) : idesc_tf32(128, PL::NQ);
      constexpr int KS = PL::O::KS;
      auto mma = [](uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
        if constexpr (BF) mma_bf16(d, a, b, id, acc);
        else mma_tf32(d, a, b, id, acc);
      };
      // failure-detection hook: a block that takes the armed request withholds
      // the completion signal of its first flux product, so that the compute
      // warps' bounded wait runs out
      bool withhold = false;
      if (P.inject && (int)blockIdx.x < ntiles && *reinterpret_cast<volatile int*>(P.inject))
        withhold = atomicExch(P.inject, 0) != 0;
      int last_k[2] = {-1, -1};   // latest staging index issued into set 0 / 1
      if ((int)blockIdx.x < ntiles) {
        stage_tile(blockIdx.x, 0);
        last_k[0] = 0;
      }
      int mit = 0;
      for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++mit) {
        if (!wait_ready(0)) { mfail = true; break; }
        if (PML) {   // V_q first: the quadrature epilogue waits for it alone
          for (int t = 0; t < PL::VQT; ++t)   // rows 128 t .. 128 t + 127
            for (int k = 0; k < NpK / KS; ++k)
              mma(tmem + PL::cVq + t * PL::NQ,
                  make_desc(sbase + PL::oVq + 16 * t * PL::SBO_V + 256 * k, 128, PL::SBO_V),
                  make_desc(sbase + PL::oBF + 2 * PL::LB * k, PL::LB, PL::SBB_V), idQ, k > 0);
          mma_commit(saddr(mbar + 0));
        }
        for (int v = 0; v < PL::VT; ++v)   // derivatives DPT v .. DPT v + DPT - 1
          for (int k = 0; k < NpK / KS; ++k)
            mma(tmem + PL::cV + v * PL::NV,
                make_desc(sbase + PL::oVol + (v * PL::DPT * Np / 8) * PL::SBO_V + 256 * k, 128,
                          PL::SBO_V),
                make_desc(sbase + PL::oBF + 2 * PL::LB * k, PL::LB, PL::SBB_V), idV, k > 0);
        issued = true;
        // the compute warps are past tile mit - 1: its staging set takes tile mit + 1
        if (tile + (int)gridDim.x < ntiles) {
          stage_tile(tile + gridDim.x, (mit + 1) & 1);
          last_k[(mit + 1) & 1] = mit + 1;
        }
        if (!wait_ready(1)) { mfail = true; break; }
        for (int k = 0; k < NFK / KS; ++k)
          mma(tmem + PL::cL, make_desc(sbase + PL::oL + 256 * k, 128, PL::SBO_L),
                   make_desc(sbase + PL::oBFL + 2 * PL::LB * k, PL::LB, PL::SBB_L), idV, k > 0);
        if (!withhold) mma_commit(saddr(mbar + 1));
        withhold = false;
        if (PML) {
          if (!wait_ready(2)) { mfail = true; break; }
          for (int k = 0; k < NqK / KS; ++k)
            mma(tmem + PL::cPq, make_desc(sbase + PL::oPq + 256 * k, 128, PL::SBO_Q),
                     make_desc(sbase + PL::oBTZ + 2 * PL::LB * k, PL::LB, PL::SBB_Q), idQ, k > 0);
          mma_commit(saddr(mbar + 2));
        }
      }
      // the staging copies this thread issued land before the memory is released
      for (int s2 = 0; s2 < 2; ++s2)
        if (last_k[s2] >= 0 && !mbar_wait(saddr(mbar + 7 + s2), (last_k[s2] >> 1) & 1))
          mfail = true;
      // every product this thread issued completes before the memory is released
      if (issued) {
        mma_commit(saddr(mbar + 6));
        if (!mbar_wait(saddr(mbar + 6), 0)) mfail = true;
      }
      // a wait that gave up, here or above, is reported as a timeout
      if (mfail) atomicExch(P.err, 1);
    }
    __syncwarp();
  } else {
  asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(TW::compute_regs));
  float Ep[FT][3], Hp[FT][3], ZPv[FT];
  int nbv[FT], codev[FT];
  float sgv[PML ? EH : 1][VQT][3];
  if ((int)blockIdx.x < ntiles) {
    load_nbr_idx(blockIdx.x, nbv, codev);
    load_nbr_val(blockIdx.x, nbv, codev, Ep, Hp, ZPv);
    load_sig(blockIdx.x, sgv);
  }

  int it = 0;
  for (int tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x, ++it) {
    const int set = it & 1;
    const int next = tile + gridDim.x;
    const float* gblk[4];
    tile_blocks(tile, gblk);
    float* SQ = staged(set, 0, gblk[0]);
    float* SR = staged(set, 1, gblk[1]);
    float* SP = PML ? staged(set, 2, gblk[2]) : nullptr;
    float* SRP = PML ? staged(set, 3, gblk[3]) : nullptr;
    const int b = tile / tiles_per_batch;
    const int t0 = (tile - b * tiles_per_batch) * T;
    const int ne = min(T, P.n_elem - t0);
    const int eg0 = P.e_begin + t0;
    const int ep0 = eg0 - P.K0;
    float* qout = P.qout + (int64_t)b * P.strideQ;
    float* resq = P.resq + (int64_t)b * P.strideQ;
    float* pio = P.p + (int64_t)b * P.strideP;
    float* resp = P.resp + (int64_t)b * P.strideP;

    if (tid == 0) flags[0] = 0;
    if (next < ntiles) {
      load_nbr_idx(next, nbv, codev);   // consumed after this tile's flux
    }
    {   // this tile's copies landed (staging use it of set it & 1)
      const bool ok = mbar_wait(saddr(mbar + 7 + set), (it >> 1) & 1);
      if (!cbar_and(kTcThreads, ok)) { failed = true; break; }
    }
    // this tile's staged geometry: normal and Fscale [T][4][4], metric
    // [T][9] (double), 1/eps, 1/mu, Z [T][3]
    const float* fn_s =
        reinterpret_cast<const float*>(staged_at(set, PL::oSFN, P.fnrm + (int64_t)eg0 * 16));
    const double* met_s =
        reinterpret_cast<const double*>(staged_at(set, PL::oSMET, P.geo + (int64_t)eg0 * 9));
    const float* mat_s =
        reinterpret_cast<const float*>(staged_at(set, PL::oSMAT, P.mat + (int64_t)eg0 * 3));
    for (int s = tid; s < P.nsrc; s += kTcThreads) {
      const int sb = s < kSrcCache ? srcc[2 * s] : P.src[s].batch;
      const int se = s < kSrcCache ? srcc[2 * s + 1] : P.src[s].elem;
      if (sb == b && se >= eg0 && se < eg0 + ne) {
        const int slot = atomicAdd(&flags[0], 1);
        if (slot < 64) srcl[slot] = s;
      }
    }
    // ---- B operand of the field products (TF32-rounded), from the staged
    // blocks: one 16-byte core-matrix row (4 consecutive nodes of one
    // (element, component) row) per task; rows of missing elements are skipped
    {
      constexpr int CW = PL::O::CW;
      constexpr int G4 = (Np + CW - 1) / CW;
      constexpr int NTASK = PL::ROWS_F * G4;
      constexpr int NIT = (NTASK + kTcThreads - 1) / kTcThreads;
      // every task's values are loaded before any is converted and stored,
      // so the loads of a thread's tasks overlap
      float x[NIT][8];
#pragma unroll
      for (int it2 = 0; it2 < NIT; ++it2) {
        const int task = tid + it2 * kTcThreads;
        const int row = task / G4, g = task - row * G4;
        const int rr = PML && row >= 6 * T ? row - 6 * T : row;
        const bool live = task < NTASK && rr < ne * 6;
        const float* src = (PML && row >= 6 * T ? SP : SQ) + rr * Np + CW * g;
#pragma unroll
        for (int h = 0; h < CW; ++h) x[it2][h] = live && CW * g + h < Np ? src[h] : 0.f;
      }
#pragma unroll
      for (int it2 = 0; it2 < NIT; ++it2) {
        const int task = tid + it2 * kTcThreads;
        const int row = task / G4, g = task - row * G4;
        const int rr = PML && row >= 6 * T ? row - 6 * T : row;
        if (task >= NTASK || rr >= ne * 6) continue;
        unsigned char* dst = smem + PL::oBF + PL::ofs(row, CW * g, PL::SBB_V, PL::LB);
        if constexpr (BF) {
          uint32_t w[4];
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            const __nv_bfloat162 v2 = __floats2bfloat162_rn(x[it2][2 * h], x[it2][2 * h + 1]);
            w[h] = *reinterpret_cast<const uint32_t*>(&v2);
          }
          *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
        } else {
          *reinterpret_cast<float4*>(dst) = make_float4(to_tf32(x[it2][0]), to_tf32(x[it2][1]),
                                                        to_tf32(x[it2][2]), to_tf32(x[it2][3]));
        }
      }
    }
    // ---- the volume and V_q products need only the field operand
    signal_ready(3);
    // ---- upwind flux, scaled by Fscale, into the B operand of LIFT
#pragma unroll
    for (int u = 0; u < FT; ++u) {
      const int task = tid + u * kTcThreads;
      if (task >= ne * NF) continue;
      const int e = task / NF, fm = task - e * NF;
      const int f = fm / Nfp;
      const int ni = Fmask[fm];
      const float* nn = fn_s + e * 16 + f * 4;
      const float nx = nn[0], ny = nn[1], nz = nn[2], fsc = nn[3];
      const float* sq = SQ + e * 6 * Np + ni;
      float Em[3], Hm[3], Eo[3], Ho[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) { Em[c] = sq[c * Np]; Hm[c] = sq[(3 + c) * Np]; }
      const float ZM = mat_s[e * 3 + 2];
      float ZP = ZPv[u];
      if (ZP < 0.f) {   // perfect electric conductor: mirror state
        ZP = ZM;
#pragma unroll
        for (int c = 0; c < 3; ++c) { Eo[c] = -Em[c]; Ho[c] = Hm[c]; }
      } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) { Eo[c] = Ep[u][c]; Ho[c] = Hp[u][c]; }
      }
      const float dEx = Eo[0] - Em[0], dEy = Eo[1] - Em[1], dEz = Eo[2] - Em[2];
      const float dHx = Ho[0] - Hm[0], dHy = Ho[1] - Hm[1], dHz = Ho[2] - Hm[2];
      const float ndE = nx * dEx + ny * dEy + nz * dEz;
      const float ndH = nx * dHx + ny * dHy + nz * dHz;
      const float cHx = ny * dHz - nz * dHy, cHy = nz * dHx - nx * dHz, cHz = nx * dHy - ny * dHx;
      const float cEx = ny * dEz - nz * dEy, cEy = nz * dEx - nx * dEz, cEz = nx * dEy - ny * dEx;
      const float al = (float)P.alpha;
      // fast division (relative error ~1e-7, far below the operand rounding)
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
      for (int c = 0; c < 6; ++c)
        put_op<BF>(smem + PL::oBFL + PL::ofs(e * 6 + c, fm, PL::SBB_L, PL::LB), fo[c]);
    }
    signal_ready(4);   // LIFT operand
    if (next < ntiles) load_nbr_val(next, nbv, codev, Ep, Hp, ZPv);
    // this tile's metric and 1/eps, 1/mu in float for the curl epilogue (read
    // after the next barrier; the previous tile's readers are past the last)
    if (tid < ne * 9) geoM[(tid / 9) * 12 + tid % 9] = (float)met_s[tid];
    if (tid < ne * 2) geoM[(tid >> 1) * 12 + 9 + (tid & 1)] = mat_s[(tid >> 1) * 3 + (tid & 1)];

    if (PML) {
      if (!wait_bar(0)) { failed = true; break; }   // V_q product
      // ---- epilogue A1: eq. 9 at the quadrature points -> B of P_q
      {
        const float ie0 = 1.f / (float)P.eps0;
#pragma unroll
        for (int t = 0; t < VQT; ++t) {       // V_q product t: points 128 t + lane row
        const uint32_t cq = PL::cVq + t * PL::NQ;
        // this lane's columns of the group's elements grp + NGRP k (warp-uniform);
        // with two per group both loads are in flight before one wait
        float vv[EH][12];
        if constexpr (EH == 2 && 2 * NGRP == T) {
          float w[24];
          tld_6x2x2(tmem + lane_base + cq + grp * 6, tmem + lane_base + cq + 6 * T + grp * 6,
                    tmem + lane_base + cq + (grp + NGRP) * 6,
                    tmem + lane_base + cq + 6 * T + (grp + NGRP) * 6, w);
#pragma unroll
          for (int i = 0; i < 12; ++i) { vv[0][i] = w[i]; vv[1][i] = w[12 + i]; }
        } else {
#pragma unroll
          for (int k = 0; k < EH; ++k) {
            const int e = grp + NGRP * k;
            if (e < T)
              tld_6x2(tmem + lane_base + cq + e * 6, tmem + lane_base + cq + 6 * T + e * 6, vv[k]);
          }
        }
#pragma unroll
        for (int k = 0; k < EH; ++k) {
          const int q = 128 * t + quad * 32 + lane;   // quadrature point of this lane
          const int e = grp + NGRP * k;
          if (e >= T) break;
          const float* v = vv[k];
          if (e >= ne || q >= NqK) continue;
          // sigma_u / eps0 at this point
          const float sg[3] = {sgv[k][t][0] * ie0, sgv[k][t][1] * ie0, sgv[k][t][2] * ie0};
          float o[12];
#pragma unroll
          for (int u = 0; u < 3; ++u) {
            const float su = sg[u], sv = sg[(u + 1) % 3], sw = sg[(u + 2) % 3];
            // eq. 9 with kappa = 1 in terms of s = sigma / eps0: a = 1,
            // b = sv + sw - su, c = sv sw - b su
            const float bc = sv + sw - su;
            const float cc = sv * sw - bc * su;
            const float dd = su;
            o[u] = bc * v[u] + cc * v[6 + u];
            o[3 + u] = bc * v[3 + u] + cc * v[9 + u];
            o[6 + u] = v[u] - dd * v[6 + u];
            o[9 + u] = v[3 + u] - dd * v[9 + u];
          }
#pragma unroll
          for (int c = 0; c < 6; ++c) {
            put_op<BF>(smem + PL::oBTZ + PL::ofs(e * 6 + c, q, PL::SBB_Q, PL::LB), o[c]);
            put_op<BF>(smem + PL::oBTZ + PL::ofs(6 * T + e * 6 + c, q, PL::SBB_Q, PL::LB), o[6 + c]);
          }
        }
        }   // t
      }
      if (next < ntiles) load_sig(next, sgv);
      signal_ready(5);   // P_q operand; the product overlaps the epilogue below
    }
    if (!wait_bar(1)) { failed = true; break; }
    const int nsrc_l = min(flags[0], 64);

    // ---- derivative and LIFT columns -> shared memory.  Lane d Np + i holds
    // the d-th derivative at node i, lane i the LIFT term at node i.
    float* DV = reinterpret_cast<float*>(smem + PL::oDV);   // [T][DVE]
    constexpr int DVE = PL::DVE;
    if constexpr (PL::VT == 1) {
      if (quad * 32 < 3 * Np) {
        const int L = quad * 32 + lane;
        const int d = L / Np, i = L - d * Np;
        // derivative d of the 6 components | LIFT of the 6 components
#pragma unroll
        for (int k = 0; k < EH; ++k) {
          const int e = grp + NGRP * k;
          if (e >= T) break;
          float v[12];
          if (quad * 32 < Np)
            tld_6x2(tmem + lane_base + PL::cV + e * 6, tmem + lane_base + PL::cL + e * 6, v);
          else
            tld6(tmem + lane_base + PL::cV + e * 6, v);
          if (e >= ne) continue;
          if (L < 3 * Np) {
#pragma unroll
            for (int c = 0; c < 6; ++c) DV[e * DVE + (c * 4 + d) * Np + i] = v[c];
          }
          if (quad * 32 < Np && L < Np) {
#pragma unroll
            for (int c = 0; c < 6; ++c) DV[e * DVE + (c * 4 + 3) * Np + i] = v[6 + c];
          }
        }
      }
    } else {
      // two derivative products: lane d Np + i of the first holds derivative d
      // (d < DPT), lane d' Np + i of the second derivative DPT + d'
      constexpr int R0 = PL::DPT * Np, R1 = (3 - PL::DPT) * Np;
      if (quad * 32 < R0) {
        const int L = quad * 32 + lane;
        const int d0 = L / Np, i0 = L - d0 * Np;
        const int d1 = PL::DPT + d0;
        for (int e = grp; e < T; e += NGRP) {
          float v[6], w[6], l[6];
          tld6(tmem + lane_base + PL::cV + e * 6, v);
          if (quad * 32 < R1) tld6(tmem + lane_base + PL::cV + PL::NV + e * 6, w);
          if (quad * 32 < Np) tld6(tmem + lane_base + PL::cL + e * 6, l);
          if (e >= ne) continue;
          if (L < R0) {
#pragma unroll
            for (int c = 0; c < 6; ++c) DV[e * DVE + (c * 4 + d0) * Np + i0] = v[c];
          }
          if (quad * 32 < R1 && L < R1) {
#pragma unroll
            for (int c = 0; c < 6; ++c) DV[e * DVE + (c * 4 + d1) * Np + i0] = w[c];
          }
          if (quad * 32 < Np && L < Np) {
#pragma unroll
            for (int c = 0; c < 6; ++c) DV[e * DVE + (c * 4 + 3) * Np + L] = l[c];
          }
        }
      }
    }
    fence_before();
    cbar_sync(kTcThreads);
    fence_after();

    // ---- epilogue A2 (all warps): curl + LIFT, rhs of E and H per (element, node)
    for (int task = tid; task < ne * Np; task += kTcThreads) {
      const int e = task / Np, i = task - e * Np;
      const int eg = eg0 + e;
      const float* dv = DV + e * DVE + i;
      const float* g = geoM + e * 12;
      float dx[6], dy[6], dz[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        const float r = dv[4 * c * Np], sd_ = dv[(4 * c + 1) * Np], t_ = dv[(4 * c + 2) * Np];
        dx[c] = g[0] * r + g[3] * sd_ + g[6] * t_;
        dy[c] = g[1] * r + g[4] * sd_ + g[7] * t_;
        dz[c] = g[2] * r + g[5] * sd_ + g[8] * t_;
      }
      float lf[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) lf[c] = dv[(4 * c + 3) * Np];
      // Cbar(H) (E rows) and Cbar(E) (H rows)
      float CH[3], CE[3];
      CH[0] = dy[5] - dz[4] + lf[0];
      CH[1] = dz[3] - dx[5] + lf[1];
      CH[2] = dx[4] - dy[3] + lf[2];
      CE[0] = dy[2] - dz[1] + lf[3];
      CE[1] = dz[0] - dx[2] + lf[4];
      CE[2] = dx[1] - dy[0] + lf[5];
      for (int s = 0; s < nsrc_l; ++s) {
        const SrcDev& sd = P.src[srcl[s]];
        if (sd.elem != eg) continue;
        const double tau = sd.width;
        const double gg = exp(-(tst - sd.t0) * (tst - sd.t0) / (4.0 * tau * tau));
        const float jt = (float)(sd.amp * (-(tst - sd.t0) / (2.0 * tau * tau)) * gg);
        const float w = P.src_w[srcl[s] * Np + i];
#pragma unroll
        for (int c = 0; c < 3; ++c) CH[c] -= jt * (float)sd.dir[c] * w;
      }
      const float ie = geoM[e * 12 + 9], im = geoM[e * 12 + 10];
      const float rhs[6] = {ie * CH[0], ie * CH[1], ie * CH[2], -im * CE[0], -im * CE[1], -im * CE[2]};
      if (!PML) {
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          const int li = (e * 6 + c) * Np + i;
          const int64_t gi = (int64_t)eg0 * 6 * Np + li;
          const float rr = rka * SR[li] + rdt * rhs[c];
          resq[gi] = rr;
          qout[gi] = SQ[li] + rkb * rr;
        }
      } else {
#pragma unroll
        for (int c = 0; c < 6; ++c) RS[(e * 6 + c) * Np + i] = rhs[c];
      }
    }

    if (PML) {
      // ---- the P_q product has had the volume/LIFT epilogue to complete
      if (!wait_bar(2)) { failed = true; break; }
      fence_async_smem();   // the (t, z) buffer is reused below
      // ---- P_q columns of the node lanes -> shared memory
      float* DP = reinterpret_cast<float*>(smem + PL::oDP);   // [T][12][Np]
      if (quad * 32 < Np) {
        const int i = quad * 32 + lane;
#pragma unroll
        for (int k = 0; k < EH; ++k) {
          const int e = grp + NGRP * k;
          if (e >= T) break;
          float v[12];   // s | rhs of P
          tld_6x2(tmem + lane_base + PL::cPq + e * 6, tmem + lane_base + PL::cPq + 6 * T + e * 6, v);
          if (e >= ne || i >= Np) continue;
#pragma unroll
          for (int k = 0; k < 12; ++k) DP[(e * 12 + k) * Np + i] = v[k];
        }
      }
      fence_before();
      cbar_sync(kTcThreads);
      fence_after();
      // ---- epilogue B (all warps): Runge-Kutta update of E, H, P^E, P^H, two
      // consecutive values of one element block per task (6 Np is even, so a
      // pair never straddles two elements and stays 8-byte aligned)
      for (int t2 = tid; t2 < ne * 3 * Np; t2 += kTcThreads) {
        const int li = 2 * t2;                  // (e * 6 + c) * Np + i
        const int e = li / (6 * Np);
        const int di = li + e * 6 * Np;         // (e * 12 + c) * Np + i
        const float2 sr = *reinterpret_cast<const float2*>(SR + li);
        const float2 sq = *reinterpret_cast<const float2*>(SQ + li);
        const float2 rs = *reinterpret_cast<const float2*>(RS + li);
        const float2 ds = *reinterpret_cast<const float2*>(DP + di);
        const float2 dz = *reinterpret_cast<const float2*>(DP + di + 6 * Np);
        const float2 srp = *reinterpret_cast<const float2*>(SRP + li);
        const float2 sp = *reinterpret_cast<const float2*>(SP + li);
        float2 rr, qn, rp, pn;
        rr.x = rka * sr.x + rdt * (rs.x - ds.x);
        rr.y = rka * sr.y + rdt * (rs.y - ds.y);
        qn.x = sq.x + rkb * rr.x;
        qn.y = sq.y + rkb * rr.y;
        rp.x = rka * srp.x + rdt * dz.x;
        rp.y = rka * srp.y + rdt * dz.y;
        pn.x = sp.x + rkb * rp.x;
        pn.y = sp.y + rkb * rp.y;
        const int64_t gi = (int64_t)eg0 * 6 * Np + li;
        const int64_t pi = (int64_t)ep0 * 6 * Np + li;
        *reinterpret_cast<float2*>(resq + gi) = rr;
        *reinterpret_cast<float2*>(qout + gi) = qn;
        *reinterpret_cast<float2*>(resp + pi) = rp;
        *reinterpret_cast<float2*>(pio + pi) = pn;
      }
    }
    fence_before();
    cbar_sync(kTcThreads);
    fence_after();
  }

  if (failed && tid == 0) atomicExch(P.err, 1);
  }   // compute warps
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) tmem_dealloc(tmem, PL::TMEM_COLS);
}

template <int N, bool PML, bool BF, int QC>
cudaError_t configure_n() {
  using TW = TcWarps<N, PML, BF, QC>;
  // the compute warps' setmaxnreg.inc waits until the block's launch
  // allocation can cover the split: refuse a build whose compiled register
  // count would leave it short
  cudaFuncAttributes fa{};
  cudaError_t e = cudaFuncGetAttributes(&fa, tc_stage_kernel<N, PML, BF, QC>);
  if (e != cudaSuccess) return e;
  if ((long)fa.numRegs * TW::threads <
      32L * TW::compute * TW::compute_regs + 32L * TW::issue * TW::issue_regs)
    return cudaErrorInvalidConfiguration;
  return cudaFuncSetAttribute(tc_stage_kernel<N, PML, BF, QC>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)Plan<N, PML, BF, QC>::bytes);
}

template <int N, bool PML, bool BF, int QC>
cudaError_t launch_n(const StageParams<float>& P, int nb, cudaStream_t s) {
  using PL = Plan<N, PML, BF, QC>;
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
  const int per_sm = PL::ONE ? 1 : 512 / (int)PL::TMEM_COLS;
  const int grid = (int)std::min<long long>(tiles, (long long)per_sm * sms);
  tc_stage_kernel<N, PML, BF, QC><<<grid, TcWarps<N, PML, BF, QC>::threads, PL::bytes, s>>>(Q);
  return cudaGetLastError();
}

}  // namespace tc

// Tensor-core stages built: TF32 operands for N <= 4 (both rules) and N = 5
// with the compact rule (its N = 5 operands with the (N+1)^3 rule do not fit
// shared memory); BF16 operands for N <= 5 with either rule.  kappa = 1.
bool tc_supported(int N, bool kappa, bool bf16, int qc) {
  if (kappa || N < 1 || N > 5) return false;
  return bf16 || N <= 4 || qc == 1;
}

// The PML class with a compact rule runs tc_rows_kernel (tc_rows.cu); here:
// the non-PML class (no quadrature) and the PML class with the (N+1)^3 rule.
template <int N, bool BF>
cudaError_t configure_tc_n() {
  cudaError_t e = cudaSuccess;
  if constexpr (BF || N <= 4) {
    e = tc::configure_n<N, false, BF, 0>();
    if (e == cudaSuccess) e = tc::configure_n<N, true, BF, 0>();
  } else {
    e = tc::configure_n<N, false, BF, 1>();
  }
  return e;
}

template <bool BF>
cudaError_t configure_tc_bf(int N) {
  switch (N) {
    case 1: return configure_tc_n<1, BF>();
    case 2: return configure_tc_n<2, BF>();
    case 3: return configure_tc_n<3, BF>();
    case 4: return configure_tc_n<4, BF>();
    case 5: return configure_tc_n<5, BF>();
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t configure_tc_kernels(int N, bool bf16) {
  return bf16 ? configure_tc_bf<true>(N) : configure_tc_bf<false>(N);
}

template <int N, bool BF>
cudaError_t launch_tc_n(bool pml, const StageParams<float>& P, int nb, cudaStream_t s, int qc) {
  if constexpr (BF || N <= 4) {
    if (!pml) return tc::launch_n<N, false, BF, 0>(P, nb, s);
    if (qc == 0) return tc::launch_n<N, true, BF, 0>(P, nb, s);
  } else {
    if (!pml) return tc::launch_n<N, false, BF, 1>(P, nb, s);
  }
  return cudaErrorInvalidValue;   // compact-rule PML classes run tc_rows_kernel
}

template <bool BF>
cudaError_t launch_tc_bf(int N, bool pml, const StageParams<float>& P, int nb, cudaStream_t s,
                         int qc) {
  switch (N) {
    case 1: return launch_tc_n<1, BF>(pml, P, nb, s, qc);
    case 2: return launch_tc_n<2, BF>(pml, P, nb, s, qc);
    case 3: return launch_tc_n<3, BF>(pml, P, nb, s, qc);
    case 4: return launch_tc_n<4, BF>(pml, P, nb, s, qc);
    case 5: return launch_tc_n<5, BF>(pml, P, nb, s, qc);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_stage_tc(int N, bool pml, const StageParams<float>& P, int nb, cudaStream_t s,
                            bool bf16, int qc) {
  // the kernels stage element blocks as bulk copies of their 16-byte-aligned
  // cover, sized for blocks that start 0 or 8 bytes past a boundary: every
  // field buffer must start on a 16-byte boundary
  const uintptr_t a = reinterpret_cast<uintptr_t>(P.qin) | reinterpret_cast<uintptr_t>(P.qout) |
                      reinterpret_cast<uintptr_t>(P.resq) |
                      (pml ? reinterpret_cast<uintptr_t>(P.p) | reinterpret_cast<uintptr_t>(P.resp)
                           : 0);
  if (a & 15) return cudaErrorMisalignedAddress;
  return bf16 ? launch_tc_bf<true>(N, pml, P, nb, s, qc)
              : launch_tc_bf<false>(N, pml, P, nb, s, qc);
}

}  // namespace wadg
