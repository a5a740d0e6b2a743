// Grouped launch of the CUDA-core stage (FP32): several contexts' element
// classes advanced by one kernel launch per Runge-Kutta stage.
#include "stage_body.cuh"

namespace wadg {

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

}  // namespace wadg
