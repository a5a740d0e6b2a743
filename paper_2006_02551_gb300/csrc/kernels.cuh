// Device-side data layout and kernel entry points of the DGTD stage.
//
// Layout in HBM (internal element order: non-PML elements first, then PML
// elements, each class in space-filling-curve order of the centroids):
//   E,H      q[b][e][6][Np]        two copies (stage input / output)
//   res      rq[b][e][6][Np]       LSERK register for E,H
//   P^E,P^H  p[b][e'][6][Np]       PML elements only (e' = e - K0), updated in place
//   res      rp[b][e'][6][Np]
//   geometry geo[e][9]             double: r_x r_y r_z s_x s_y s_z t_x t_y t_z
//            geof[e][9]            the same in float (tensor-core contexts)
//            fnrm[e][4][4]         unit outward normal and Fscale = sJ/J per face
//                                  (computed in double on the host)
//   material mat[e][3]             1/eps, 1/mu, Z = sqrt(mu/eps)
//   faces    nbr[e][4] (-1: PEC), code[e][4] = neighbour face * 6 + rotation
//   PML      sig[e'][3][Nq] (and kap[e'][3][Nq])  sigma_u, kappa_u at the
//            quadrature nodes of each PML element (weight-adjusted scheme;
//            with element-constant coefficients every node holds the value
//            at the centroid)
//            stored[e'][3][3][Np][NpP]  stored-matrix scheme: per axis u the
//            operators M_k^-1 M_k^{b_u}, M_k^-1 M_k^{c_u}, M_k^-1 M_k^{d_u},
//            transposed (column j of the operator is row j here)
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace wadg {

// Checked builds (-DWADG_CHECKED, a diagnostic build of the library): index
// checks before the scattered reads of the stage kernels record a violation
// in the context's status word (value 2) and skip the read; in other builds
// WADG_INDEX_OK is the constant true and costs nothing.
#ifdef WADG_CHECKED
__device__ __forceinline__ bool wadg_index_ok(bool ok, int* status) {
  if (!ok) atomicOr(status, 2);
  return ok;
}
#define WADG_INDEX_OK(cond, status) ::wadg::wadg_index_ok((cond), (status))
#else
#define WADG_INDEX_OK(cond, status) true
#endif

// Volume quadrature capacity of the PML stage kernels (eqs. 20, 21, 26-29).
// Class 0: the default conical-product rule of (N+1)^3 points.  Class 1:
// compact rules of degree 2N of at most compact_nq(N) points (a rule with
// fewer points is padded with zero-weight points).  The kernels are compiled
// for both classes; the context picks one from the size of its rule.
__host__ __device__ constexpr int compact_nq(int N) {
  return N == 1 ? 4 : N == 2 ? 14 : N == 3 ? 24 : N == 4 ? 48 : N == 5 ? 84 : 0;
}
__host__ __device__ constexpr int quad_capacity(int N, int qc) {
  return qc ? compact_nq(N) : (N + 1) * (N + 1) * (N + 1);
}

struct SrcDev {
  int elem;     // internal element id
  int batch;
  double dir[3];
  double t0, width, amp;
};

template <typename Real>
struct StageParams {
  const Real* qin;
  Real* qout;
  Real* resq;
  Real* p;
  Real* resp;
  Real* pout;               // P after the stage (null: in place over p; CUDA-core kernels)
  const double* geo;
  const float* geof;        // [e][9]: the metric in float (tensor-core contexts)
  const Real* fnrm;         // [e][4][4]: unit outward normal, Fscale (from FP64)
  const Real* mat;
  const int* nbr;
  const unsigned char* code;
  const Real* sig;
  const Real* kap;
  const Real* stored;       // stored-matrix operators (stored-matrix scheme only)
  const Real* ops;          // DrT | DsT | DtT | LIFTT | VqT | PqT
  const unsigned char* tabs;  // Fmask[4 Nfp] | fperm[4*24*Nfp]
  int64_t strideQ;          // elements*6*Np per batch (all elements)
  int64_t strideP;          // K1*6*Np per batch
  int K0;                   // first PML element (internal id)
  int e_begin;              // first element of this launch's class
  int n_elem;               // elements of this launch's class
  int nb;                   // excitations (set by the launcher)
  int tile_elems;           // CUDA-core kernels: elements per tile (0: the largest that fits)
  int nsrc;
  const SrcDev* src;
  const Real* src_w;        // [nsrc][Np]: M_k^{-1} l(r_s)
  double rk_a, rk_b, rk_c, dt;
  double t;                 // base time if t_dev == nullptr
  const double* t_dev;      // device base time (graph replays)
  double eps0;
  double alpha;             // flux upwinding (1 upwind, 0 central)
  const void* tcops;        // tensor-core operator tables (TF32 path)
  int* err;                 // device error flag (bounded waits that gave up)
  int* inject;              // tensor-core kernels: armed failure-detection request
                            // (nonzero: one block withholds a product signal), or null
};

// reverse Runge-Kutta stage (adjoint.cu)
template <typename Real>
struct AdjParams {
  Real* lam_q;              // adjoint of E,H [b][e][6][Np], updated in place
  Real* rho_q;              // adjoint of the E,H register
  Real* lam_p;              // adjoint of P [b][e'][6][Np]
  Real* rho_p;
  const Real* q_in;         // forward stage input (E,H)
  const Real* p_in;         // forward stage input (P)
  Real* G;                  // scratch [b][e][4 Nfp][6]
  double* grad_eps;         // [b][K] internal order
  double* grad_prof;        // [b][6]: d/dsigma_max[3], d/dp_sigma[3]
  const double* geo;
  const Real* fnrm;         // [e][4][4]: unit outward normal, Fscale (as the forward stage)
  const Real* mat;
  const int* nbr;
  const unsigned char* code;
  const Real* sig;
  const Real* ops;
  const Real* adj_ops;      // Dr, Ds, Dt [Np][NpP], LIFT [Np][NFP], P_q [Np][NqP], V_q [Nq][NpP]
  const unsigned char* tabs;
  int64_t strideQ, strideP;
  int K, K0, e_begin, n_elem;
  int nsrc;
  const SrcDev* src;
  const Real* src_w;
  double rk_a, rk_b, dt, t, eps0, alpha;
  double sigma_max[3], p_sigma[3];
  Real inv_sigma_max[3], inv_p_sigma[3];   // 1 / sigma_max, 1 / p_sigma (0 where unset)
  // the same scalars rounded once on the host (no per-thread conversion)
  Real rk_a_r, rk_b_r, dt_r, alpha_r, inv_eps0_r;
};

struct ProbeParams {
  const void* q;            // current E,H
  int64_t strideQ;
  int nprobe, nb, Np;
  const int* elem;          // [nprobe]
  const double* ell;        // [nprobe][Np]
  double* out;              // [nsteps][nprobe][6][nb]
  double* obj;              // [nb]
  const int64_t* step;      // device step counter since run start
};

// launchers (return cudaError_t of the launch)
// qc: quadrature class of the PML kernels (quad_capacity)
template <typename Real>
cudaError_t configure_stage_kernels(int N);  // once per device, outside graph capture
template <typename Real>
cudaError_t launch_stage(int N, bool pml, bool kappa, const StageParams<Real>& P, int nb,
                         cudaStream_t s, int qc = 0);
cudaError_t launch_probes(bool fp64, const ProbeParams& P, cudaStream_t s);
template <typename Real>
cudaError_t configure_adjoint_kernels(int N);
template <typename Real>
cudaError_t launch_adjoint_stage(int N, const AdjParams<Real>& P, int nb, cudaStream_t s,
                                 int qc = 0);
template <typename Real>
cudaError_t launch_adjoint_probes(const Real* q, int64_t strideQ, int nprobe, int nb, int Np,
                                  const int* elem, const double* ell, Real* lam, cudaStream_t s);
// tensor-core (tcgen05) stage kernels: TF32 operands, or BF16 operands (bf16)
// tc_supported: whether a tensor-core stage exists for (N, bf16, qc)
bool tc_supported(int N, bool kappa, bool bf16, int qc = 0);
cudaError_t configure_tc_kernels(int N, bool bf16);
cudaError_t launch_stage_tc(int N, bool pml, const StageParams<float>& P, int nb, cudaStream_t s,
                            bool bf16, int qc = 0);
// row-owned tensor-core PML stage kernels (compact volume rules)
cudaError_t configure_tc_rows(int N, bool bf16);
cudaError_t launch_pml_tc_rows(int N, const StageParams<float>& P, int nb, cudaStream_t s,
                               bool bf16);
cudaError_t launch_advance(double* t_dev, int64_t* step_dev, double dt, cudaStream_t s);
template <typename Real>
cudaError_t launch_pml_samples(int Nq, int K1, int K0, const double* verts,
                               const double* rq /*[Nq][3]*/, const double* prof /*16*/,
                               Real* sig, Real* kap, bool element_constant, cudaStream_t s);
// stored-matrix scheme: the PML class with the per-element operators (3 per
// axis with kappa = 1: B, C, D; 5 otherwise: B, C, D, K = M^-1 M^{1/kappa},
// A^-1 = (M^a)^-1 M), and their construction in double precision from the
// sigma and kappa profiles at the points of a high-degree rule (rh [Nh][3]
// reference points, Ph [Np][Nh] = M^-1 V_h^T W_h, Vh [Nh][Np]; prof as for
// launch_pml_samples; *bad set if an a_u operator has a zero pivot)
template <typename Real>
cudaError_t launch_stage_stored(int N, bool kappa, const StageParams<Real>& P, int nb,
                                cudaStream_t s);
template <typename Real>
cudaError_t configure_stored_kernels(int N);
template <typename Real>
cudaError_t launch_stored_ops(int N, int K1, int K0, const double* verts, const double* prof,
                              const double* rh, const double* Ph, const double* Vh, int Nh,
                              bool kappa, Real* out, int* bad, cudaStream_t s);
// grouped launch (FP32 CUDA-core kernels): item i runs order code[i] / 4 with
// class code[i] % 4 (0 non-PML, 1 PML, 2 PML with kappa); blocks
// [first[i], first[i+1]) start on item i, and every block takes tiles from
// counter[i] (zeroed before the launch) until all ntiles[i] are taken, then
// moves on to the next item with tiles left
// the items of one variant (order, element class) of a group
struct GroupParams {
  const StageParams<float>* p;   // [nitems], device memory
  const int* first;              // [nitems + 1] static block split, device memory
  const int* ntiles;             // [nitems], device memory
  int* counter;                  // [nitems], device memory
  int nitems;
};
cudaError_t configure_group_kernel();
// dynamic shared memory and largest tile (elements) of one item; threads per
// block, blocks per SM and launch of the kernel of variant code = N * 4 +
// (0 non-PML, 1 PML, 2 PML with kappa)
size_t group_smem_bytes(int N, bool pml, int tile);
int group_tile_max(int N, bool pml);
int group_threads(int code);
int group_blocks_per_sm(int code, size_t smem);
cudaError_t launch_group_stage(int code, const GroupParams& G, int nblocks, size_t smem,
                               cudaStream_t s);
template <typename Real>
cudaError_t launch_check_finite(const Real* a, int64_t n, int* flag, cudaStream_t s);
// state exchange between a caller's device array user[nb][K][12][Np] (double,
// caller element order, perm[internal] = caller id) and the internal E,H and
// P blocks; to_internal selects the direction (P of non-PML elements: ignored
// / written as zero)
template <typename Real>
cudaError_t launch_state_exchange(bool to_internal, const int* perm, int64_t K, int64_t K0,
                                  int Np, int nb, double* user, Real* q, Real* p,
                                  cudaStream_t s);

}  // namespace wadg
