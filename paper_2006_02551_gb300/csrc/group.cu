// Grouped launch of the CUDA-core stage (FP32): several contexts' element
// classes advanced with one launch per (order, element class) variant and
// Runge-Kutta stage.
#include "stage_body.cuh"

namespace wadg {

// ------------------------------------------------------------ grouped launch
// A grouped stage advances every element class of every context of a group
// by one stage (FP32) with one launch per (order, element class) variant
// present.  A variant's kernel is the single-context stage kernel of that
// variant (same body, block shape, tile and register budget) with a dynamic
// tile schedule over the variant's items; the host issues a stage's variant
// launches on parallel branches of the step graph, so one variant's blocks
// take the SMs that another's leave as its tiles run out.

template <int N, bool PML>
using GTile = Tile<float, N, PML, 0, 0>;

// dynamic shared memory of one item with `tile` elements per tile
template <int N, bool PML>
size_t group_smem_one(int tile) {
  using TL = GTile<N, PML>;
  const int t = tile > 0 && tile < TL::T ? tile : TL::T;
  return (size_t)(TL::ops_sz + t * TL::per_elem) * sizeof(float) + 64 * sizeof(int);
}

size_t group_smem_bytes(int N, bool pml, int tile) {
  switch (N) {
    case 1: return pml ? group_smem_one<1, true>(tile) : group_smem_one<1, false>(tile);
    case 2: return pml ? group_smem_one<2, true>(tile) : group_smem_one<2, false>(tile);
    case 3: return pml ? group_smem_one<3, true>(tile) : group_smem_one<3, false>(tile);
    case 4: return pml ? group_smem_one<4, true>(tile) : group_smem_one<4, false>(tile);
    case 5: return pml ? group_smem_one<5, true>(tile) : group_smem_one<5, false>(tile);
    default: return 0;
  }
}

int group_tile_max(int N, bool pml) {
  switch (N) {
    case 1: return pml ? GTile<1, true>::T : GTile<1, false>::T;
    case 2: return pml ? GTile<2, true>::T : GTile<2, false>::T;
    case 3: return pml ? GTile<3, true>::T : GTile<3, false>::T;
    case 4: return pml ? GTile<4, true>::T : GTile<4, false>::T;
    case 5: return pml ? GTile<5, true>::T : GTile<5, false>::T;
    default: return 0;
  }
}

// every block starts on the item of the variant that the static split gives
// it, takes that item's tiles from its counter, then moves on to the
// variant's items that still have tiles
template <int N, bool PML, bool KAPPA>
__global__ void __launch_bounds__(GTile<N, PML>::THREADS) group_stage_kernel(const GroupParams G) {
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
    stage_body<float, N, PML, KAPPA, false, 0>(P, smem_raw, 0, 1, G.counter + it);
  }
}

// variant code = N * 4 + (0 non-PML, 1 PML, 2 PML with kappa); f receives
// the kernel and its threads per block
template <typename F>
cudaError_t with_variant(int code, F&& f) {
#define WADG_GROUP_CASE(NN)                                                             \
  case NN * 4 + 0: return f(group_stage_kernel<NN, false, false>, GTile<NN, false>::THREADS); \
  case NN * 4 + 1: return f(group_stage_kernel<NN, true, false>, GTile<NN, true>::THREADS);   \
  case NN * 4 + 2: return f(group_stage_kernel<NN, true, true>, GTile<NN, true>::THREADS);
  switch (code) {
    WADG_GROUP_CASE(1)
    WADG_GROUP_CASE(2)
    WADG_GROUP_CASE(3)
    WADG_GROUP_CASE(4)
    WADG_GROUP_CASE(5)
    default: return cudaErrorInvalidValue;
  }
#undef WADG_GROUP_CASE
}

cudaError_t configure_group_kernel() {
  for (int N = 1; N <= 5; ++N)
    for (int v = 0; v < 3; ++v) {
      const size_t smem = group_smem_bytes(N, v > 0, 0);
      cudaError_t e = with_variant(N * 4 + v, [&](auto k, int) {
        return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      });
      if (e != cudaSuccess) return e;
    }
  return cudaSuccess;
}

int group_threads(int code) {
  int t = 0;
  with_variant(code, [&](auto, int threads) {
    t = threads;
    return cudaSuccess;
  });
  return t;
}

int group_blocks_per_sm(int code, size_t smem) {
  int nb = 0;
  cudaError_t e = with_variant(code, [&](auto k, int threads) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, threads, smem);
  });
  if (e != cudaSuccess || nb < 1) nb = 1;
  return nb;
}

cudaError_t launch_group_stage(int code, const GroupParams& G, int nblocks, size_t smem,
                               cudaStream_t s) {
  if (nblocks <= 0 || G.nitems <= 0) return cudaSuccess;
  cudaError_t e = with_variant(code, [&](auto k, int threads) {
    k<<<nblocks, threads, smem, s>>>(G);
    return cudaSuccess;
  });
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace wadg
