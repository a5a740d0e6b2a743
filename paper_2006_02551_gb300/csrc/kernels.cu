// DGTD stage kernels for sm_103a: one fused launch per element class and
// Runge-Kutta stage computes the right-hand side of the semi-discrete
// system and applies the low-storage Runge-Kutta update (the stage body is in
// stage_body.cuh); probes, clocks and set-up kernels.
#include "stage_body.cuh"

namespace wadg {

template <typename Real, int N, bool PML, bool KAPPA, bool STORED = false, int QC = 0>
__global__ void __launch_bounds__(Tile<Real, N, PML, 0, QC>::THREADS)
stage_kernel(const StageParams<Real> P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  stage_body<Real, N, PML, KAPPA, STORED, 0, QC>(P, smem_raw, blockIdx.x, gridDim.x);
}

template <typename Real, int N, bool PML, bool KAPPA, bool STORED = false, int QC = 0>
static cudaError_t configure_one() {
  using TL = Tile<Real, N, PML, 0, QC>;
  return cudaFuncSetAttribute(stage_kernel<Real, N, PML, KAPPA, STORED, QC>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TL::smem);
}

// resident blocks per SM of one stage-kernel instance (cached per instance)
template <typename Real, int N, bool PML, bool KAPPA, bool STORED = false, int QC = 0>
static int resident_blocks() {
  static int cached = 0;
  if (cached == 0) {
    using TL = Tile<Real, N, PML, 0, QC>;
    int nb = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &nb, stage_kernel<Real, N, PML, KAPPA, STORED, QC>, TL::THREADS, TL::smem) !=
            cudaSuccess ||
        nb < 1)
      nb = 1;
    cached = nb * (sms > 0 ? sms : 1);
  }
  return cached;
}

template <typename Real, int N, bool PML, bool KAPPA, bool STORED = false, int QC = 0>
static cudaError_t launch_one(const StageParams<Real>& P, int nb, cudaStream_t s) {
  using TL = Tile<Real, N, PML, 0, QC>;
  if (P.n_elem <= 0) return cudaSuccess;
  StageParams<Real> Q = P;
  Q.nb = nb;
  const long long tiles = (long long)((P.n_elem + TL::T - 1) / TL::T) * nb;
  const int grid =
      (int)std::min<long long>(tiles, resident_blocks<Real, N, PML, KAPPA, STORED, QC>());
  stage_kernel<Real, N, PML, KAPPA, STORED, QC><<<grid, TL::THREADS, TL::smem, s>>>(Q);
  return cudaGetLastError();
}

template <typename Real, int N>
static cudaError_t configure_n() {
  cudaError_t e = configure_one<Real, N, false, false>();
  if (e == cudaSuccess) e = configure_one<Real, N, true, false>();
  if (e == cudaSuccess) e = configure_one<Real, N, true, true>();
  if (e == cudaSuccess) e = configure_one<Real, N, true, false, false, 1>();
  if (e == cudaSuccess) e = configure_one<Real, N, true, true, false, 1>();
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
                                cudaStream_t s, int qc) {
  if (!pml) return launch_one<Real, N, false, false>(P, nb, s);
  if (qc) {
    if (kappa) return launch_one<Real, N, true, true, false, 1>(P, nb, s);
    return launch_one<Real, N, true, false, false, 1>(P, nb, s);
  }
  if (kappa) return launch_one<Real, N, true, true>(P, nb, s);
  return launch_one<Real, N, true, false>(P, nb, s);
}

template <typename Real>
cudaError_t launch_stage(int N, bool pml, bool kappa, const StageParams<Real>& P, int nb,
                         cudaStream_t s, int qc) {
  switch (N) {
    case 1: return dispatch_pml<Real, 1>(pml, kappa, P, nb, s, qc);
    case 2: return dispatch_pml<Real, 2>(pml, kappa, P, nb, s, qc);
    case 3: return dispatch_pml<Real, 3>(pml, kappa, P, nb, s, qc);
    case 4: return dispatch_pml<Real, 4>(pml, kappa, P, nb, s, qc);
    case 5: return dispatch_pml<Real, 5>(pml, kappa, P, nb, s, qc);
    default: return cudaErrorInvalidValue;
  }
}
template cudaError_t launch_stage<double>(int, bool, bool, const StageParams<double>&, int,
                                          cudaStream_t, int);
template cudaError_t launch_stage<float>(int, bool, bool, const StageParams<float>&, int,
                                         cudaStream_t, int);

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

// State exchange with a caller's device array in the layout of the C ABI,
// user[b][k][12][Np] (double, caller element order k = perm[e]), against the
// internal E,H blocks q[b][e][6][Np] and P blocks p[b][e - K0][6][Np]
// (Real).  One thread per (b, e, component, node); consecutive threads walk
// the nodes of one internal block (contiguous on both sides).
template <typename Real>
__global__ void state_exchange_kernel(bool to_internal, const int* perm, int64_t K, int64_t K0,
                                      int Np, int nb, double* user, Real* q, Real* p) {
  const int64_t n = (int64_t)nb * K * 12 * Np;
  const int64_t K1 = K - K0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int node = (int)(i % Np);
    int64_t r = i / Np;
    const int c = (int)(r % 12);
    r /= 12;
    const int64_t e = r % K;
    const int64_t b = r / K;
    double* u = user + ((b * K + perm[e]) * 12 + c) * Np + node;
    Real* in = nullptr;
    if (c < 6) in = q + ((b * K + e) * 6 + c) * Np + node;
    else if (e >= K0) in = p + ((b * K1 + (e - K0)) * 6 + (c - 6)) * Np + node;
    if (to_internal) {
      if (in) *in = (Real)*u;
    } else {
      *u = in ? (double)*in : 0.0;
    }
  }
}

template <typename Real>
cudaError_t launch_state_exchange(bool to_internal, const int* perm, int64_t K, int64_t K0,
                                  int Np, int nb, double* user, Real* q, Real* p,
                                  cudaStream_t s) {
  const int64_t n = (int64_t)nb * K * 12 * Np;
  if (n == 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 8);
  state_exchange_kernel<Real><<<(unsigned)blocks, 256, 0, s>>>(to_internal, perm, K, K0, Np, nb,
                                                               user, q, p);
  return cudaGetLastError();
}
template cudaError_t launch_state_exchange<double>(bool, const int*, int64_t, int64_t, int, int,
                                                   double*, double*, double*, cudaStream_t);
template cudaError_t launch_state_exchange<float>(bool, const int*, int64_t, int64_t, int, int,
                                                  double*, float*, float*, cudaStream_t);

}  // namespace wadg
