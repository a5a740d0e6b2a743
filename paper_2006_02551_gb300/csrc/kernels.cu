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
template <typename Real, int N>
static cudaError_t configure_stored_n() {
  cudaError_t e = configure_one<Real, N, true, false, true>();
  if (e == cudaSuccess) e = configure_one<Real, N, true, true, true>();
  return e;
}

template <typename Real>
cudaError_t configure_stored_kernels(int N) {
  switch (N) {
    case 1: return configure_stored_n<Real, 1>();
    case 2: return configure_stored_n<Real, 2>();
    case 3: return configure_stored_n<Real, 3>();
    case 4: return configure_stored_n<Real, 4>();
    case 5: return configure_stored_n<Real, 5>();
    default: return cudaErrorInvalidValue;
  }
}
template cudaError_t configure_stored_kernels<double>(int);
template cudaError_t configure_stored_kernels<float>(int);

template <typename Real, int N>
static cudaError_t launch_stored_n(bool kappa, const StageParams<Real>& P, int nb, cudaStream_t s) {
  return kappa ? launch_one<Real, N, true, true, true>(P, nb, s)
               : launch_one<Real, N, true, false, true>(P, nb, s);
}

template <typename Real>
cudaError_t launch_stage_stored(int N, bool kappa, const StageParams<Real>& P, int nb,
                                cudaStream_t s) {
  switch (N) {
    case 1: return launch_stored_n<Real, 1>(kappa, P, nb, s);
    case 2: return launch_stored_n<Real, 2>(kappa, P, nb, s);
    case 3: return launch_stored_n<Real, 3>(kappa, P, nb, s);
    case 4: return launch_stored_n<Real, 4>(kappa, P, nb, s);
    case 5: return launch_stored_n<Real, 5>(kappa, P, nb, s);
    default: return cudaErrorInvalidValue;
  }
}
template cudaError_t launch_stage_stored<double>(int, bool, const StageParams<double>&, int,
                                                 cudaStream_t);
template cudaError_t launch_stage_stored<float>(int, bool, const StageParams<float>&, int,
                                                cudaStream_t);

// Stored operators M_k^-1 M_k^{alpha} = P_h diag(alpha(x_h)) V_h of eq. 15 for
// the coefficients alpha of eq. 9 on each axis u = x, y, z, of TE elements per
// block, in double precision.  Kinds per axis: 0 b_u, 1 c_u, 2 d_u, and with
// kappa != 1 also 3 kappa_u^-1 and 4 a_u (the last is inverted in place by
// stored_invert_kernel).  A launch computes the kinds of one set (0: b, c, d;
// 1: kappa^-1, a).  The rule's points are processed in chunks staged in shared
// memory (P_h and V_h columns, the coefficient samples of each element); every
// thread accumulates ENT entries (i, j) of the set's operators of each of its
// block's elements in registers.  Layout: block (e, u, kind) at
// ((e * 3 + u) * NB + kind) * Np * NpP, transposed (entry (i, j) at j NpP + i),
// NB = 3 kinds (kappa = 1) or 5.
template <int N>
struct StoredSetup {
  static constexpr int Np = (N + 1) * (N + 2) * (N + 3) / 6;
  static constexpr int NpP = (Np + 3) & ~3;
  static constexpr int THREADS = 256;
  static constexpr int ENT = (Np * Np + THREADS - 1) / THREADS;
  static constexpr int TE = ENT <= 2 ? 4 : (ENT <= 5 ? 2 : 1);
  static constexpr int HC = 32;
};

template <typename Real, int N, int SET>
__global__ void __launch_bounds__(StoredSetup<N>::THREADS)
stored_ops_kernel(int K1, int K0, int Nh, const double* verts, const double* prof,
                  const double* rh, const double* Ph, const double* Vh, int NB, Real* out) {
  using S = StoredSetup<N>;
  constexpr int Np = S::Np, NpP = S::NpP, NT = S::THREADS, ENT = S::ENT, TE = S::TE, HC = S::HC;
  constexpr int NK = SET == 0 ? 3 : 2;   // kinds of this set
  constexpr int K0K = SET == 0 ? 0 : 3;  // first kind of this set
  constexpr int NM = 3 * NK;
  __shared__ double PhC[Np][HC];
  __shared__ double VhC[HC][Np];
  __shared__ double al[TE][NM][HC];   // [element][NK u + kind][point]
  const int tid = threadIdx.x;
  const int e0 = blockIdx.x * TE;
  double acc[TE][NM][ENT];
#pragma unroll
  for (int t = 0; t < TE; ++t)
#pragma unroll
    for (int m = 0; m < NM; ++m)
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
      double sg[3] = {0.0, 0.0, 0.0}, kp[3] = {1.0, 1.0, 1.0};
      if (e0 + t < K1 && h0 + hh < Nh) {
        const double* v = verts + (int64_t)(K0 + e0 + t) * 12;
        const double r = rh[(h0 + hh) * 3], s_ = rh[(h0 + hh) * 3 + 1], tt = rh[(h0 + hh) * 3 + 2];
        const double l0 = -0.5 * (1 + r + s_ + tt), l1 = 0.5 * (1 + r), l2 = 0.5 * (1 + s_),
                     l3 = 0.5 * (1 + tt);
        for (int u = 0; u < 3; ++u) {
          const double x = l0 * v[u] + l1 * v[3 + u] + l2 * v[6 + u] + l3 * v[9 + u];
          const double d = (fabs(x) - prof[u]) / prof[3 + u];
          const double g = d > 0 ? pow(d, prof[9 + u]) : 0.0;
          sg[u] = d > 0 ? prof[6 + u] * g : 0.0;
          kp[u] = 1.0 + (prof[12 + u] - 1.0) * g;   // 1 exactly where d <= 0 or kappa_max = 1
        }
      }
      for (int u = 0; u < 3; ++u) {
        const int v_ = (u + 1) % 3, w_ = (u + 2) % 3;
        const double su = sg[u], sv = sg[v_], sw = sg[w_];
        const double ku = kp[u], kv = kp[v_], kw = kp[w_];
        const double a = kv * kw / ku;                       // eq. 9
        if (SET == 0) {
          const double b = (sv * kw + sw * kv - a * su) * ie0 / ku;
          al[t][3 * u][hh] = b;
          al[t][3 * u + 1][hh] = sv * sw * ie0 * ie0 - b * su * ie0;
          al[t][3 * u + 2][hh] = su * ie0 / ku;
        } else {
          al[t][2 * u][hh] = 1.0 / ku;
          al[t][2 * u + 1][hh] = a;
        }
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
          for (int m = 0; m < NM; ++m) acc[t][m][k] += w * al[t][m][hh];
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
      for (int m = 0; m < NM; ++m) {   // transposed: row j of the stored block is column j
        const int u = m / NK, kind = K0K + m % NK;
        out[((((int64_t)(e0 + t) * 3 + u) * NB + kind) * Np + j) * NpP + i] = (Real)acc[t][m][k];
      }
    }
  }
}

// In place, the inverse of the stored a_u operator A = M_k^-1 M_k^{a_u} (kind
// 4) of every element and axis, so that the stage applies A^-1 =
// (M_k^{a_u})^-1 M_k of eqs. 10, 11: Gauss-Jordan elimination with partial
// pivoting on [A | I] in double precision, one block per (element, axis).
// A zero pivot (A is similar to a positive definite matrix, so none should
// occur) sets *bad.
template <typename Real, int N>
__global__ void __launch_bounds__(128) stored_invert_kernel(int K1, Real* ops, int* bad) {
  constexpr int Np = (N + 1) * (N + 2) * (N + 3) / 6;
  constexpr int NpP = (Np + 3) & ~3;
  constexpr int W = 2 * Np;
  constexpr int NT = 128;
  extern __shared__ double Msh[];   // [Np][W]
  __shared__ double fac[Np];
  __shared__ int piv;
  __shared__ double pivv;
  const int tid = threadIdx.x, lane = tid & 31;
  const int64_t eu = blockIdx.x;    // element * 3 + axis
  if (eu >= 3 * (int64_t)K1) return;
  Real* blk = ops + (eu * 5 + 4) * Np * NpP;
  for (int idx = tid; idx < Np * Np; idx += NT) {
    const int i = idx / Np, j = idx - i * Np;
    Msh[i * W + j] = (double)blk[j * NpP + i];
    Msh[i * W + Np + j] = i == j ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int k = 0; k < Np; ++k) {
    if (tid < 32) {   // pivot: the largest |A[i][k]|, i >= k (the first of equals)
      double best = -1.0;
      int bi = k;
      for (int i = k + lane; i < Np; i += 32) {
        const double v = fabs(Msh[i * W + k]);
        if (v > best) { best = v; bi = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) piv = bi;
    }
    __syncthreads();
    const int pk = piv;
    if (pk != k)
      for (int j = tid; j < W; j += NT) {
        const double t = Msh[k * W + j];
        Msh[k * W + j] = Msh[pk * W + j];
        Msh[pk * W + j] = t;
      }
    __syncthreads();
    if (tid == 0) {
      pivv = Msh[k * W + k];
      if (!(fabs(pivv) > 1e-300)) {
        atomicExch(bad, 1);
        pivv = 1.0;
      }
    }
    __syncthreads();
    for (int j = tid; j < W; j += NT) Msh[k * W + j] /= pivv;
    for (int i = tid; i < Np; i += NT) fac[i] = i == k ? 0.0 : Msh[i * W + k];
    __syncthreads();
    for (int idx = tid; idx < Np * W; idx += NT) {
      const int i = idx / W, j = idx - i * W;
      Msh[idx] -= fac[i] * Msh[k * W + j];
    }
    __syncthreads();
  }
  for (int idx = tid; idx < Np * Np; idx += NT) {
    const int i = idx / Np, j = idx - i * Np;
    blk[j * NpP + i] = (Real)Msh[i * W + Np + j];
  }
}

template <typename Real>
cudaError_t launch_stored_ops(int N, int K1, int K0, const double* verts, const double* prof,
                              const double* rh, const double* Ph, const double* Vh, int Nh,
                              bool kappa, Real* out, int* bad, cudaStream_t s) {
  if (K1 <= 0) return cudaSuccess;
  const int NB = kappa ? 5 : 3;
#define WADG_STORED_CASE(NN)                                                              \
  case NN: {                                                                              \
    using S = StoredSetup<NN>;                                                            \
    const int grid = (K1 + S::TE - 1) / S::TE;                                            \
    stored_ops_kernel<Real, NN, 0><<<grid, S::THREADS, 0, s>>>(K1, K0, Nh, verts, prof,   \
                                                               rh, Ph, Vh, NB, out);      \
    if (kappa) {                                                                          \
      stored_ops_kernel<Real, NN, 1><<<grid, S::THREADS, 0, s>>>(K1, K0, Nh, verts, prof, \
                                                                 rh, Ph, Vh, NB, out);    \
      constexpr int Np = S::Np;                                                           \
      const size_t sm = (size_t)Np * 2 * Np * sizeof(double);                             \
      cudaError_t e = cudaFuncSetAttribute(stored_invert_kernel<Real, NN>,                \
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                           (int)sm);                                      \
      if (e != cudaSuccess) return e;                                                     \
      stored_invert_kernel<Real, NN><<<3 * K1, 128, sm, s>>>(K1, out, bad);               \
    }                                                                                     \
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
                                               bool, double*, int*, cudaStream_t);
template cudaError_t launch_stored_ops<float>(int, int, int, const double*, const double*,
                                              const double*, const double*, const double*, int,
                                              bool, float*, int*, cudaStream_t);

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
