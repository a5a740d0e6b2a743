// C ABI: context, host set-up (FP64 geometry, face connectivity, element
// classing and ordering), device uploads and the stepping loop.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/wadg.h"
#include "kernels.cuh"
#include "refelem.hpp"

using namespace wadg;

namespace {
thread_local std::string g_err;

// LSERK(5,4) coefficients (Carpenter & Kennedy); the stage times are the
// times at which each stage samples the right-hand side, obtained by running
// the recursion on y' = 1.
const double kRkA[5] = {0.0, -567301805773.0 / 1357537059087.0,
                        -2404267990393.0 / 2016746695238.0,
                        -3550918686646.0 / 2091501179385.0,
                        -1275806237668.0 / 842570457699.0};
const double kRkB[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                        1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                        2277821191437.0 / 14882151754819.0};
struct RkC {
  double c[5];
  RkC() {
    double y = 0.0, res = 0.0;
    for (int i = 0; i < 5; ++i) {
      c[i] = y;
      res = kRkA[i] * res + 1.0;
      y += kRkB[i] * res;
    }
  }
};
const RkC kRkC;

// Device bytes a context may hold (limit 0: no cap) and holds.  The
// allocations made while one of the context's entry points runs count
// against it (see BudgetScope).
struct Budget {
  size_t limit = 0, held = 0;
};
thread_local Budget* t_budget = nullptr;
struct BudgetScope {
  Budget* prev;
  explicit BudgetScope(Budget* b) : prev(t_budget) { t_budget = b; }
  ~BudgetScope() { t_budget = prev; }
};

struct DevPtr {
  void* p = nullptr;
  size_t bytes = 0;
  Budget* owner = nullptr;   // budget the bytes count against, if any
  bool borrowed = false;     // points into caller memory (wadg_bind_state)
};

}  // namespace

struct wadg_ctx {
  int N = 0;
  wadg_precision prec = WADG_FP64;
  int nb = 1;
  int device = 0;
  cudaStream_t stream = nullptr;
  // branch of the step graphs: the non-PML class of a stage runs on it, beside
  // the PML class on `stream` (created at the first capture)
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool own_stream = false;
  std::string err;
  RefOps ref;
  size_t rs = 8;  // bytes per Real

  // user-order host mesh data
  bool has_mesh = false;
  int64_t K = 0, nv = 0;
  std::vector<double> vxyz;
  std::vector<int64_t> etov;
  std::vector<double> eps_r, mu_r;
  std::vector<int64_t> nbr_u;   // [K][4] neighbour (user id) or -1
  std::vector<int> code_u;      // [K][4] neighbour face*6 + rotation
  std::vector<double> metric_u; // [K][9]
  std::vector<double> J_u;
  double fscale_max = 0.0;

  bool has_prof = false;
  wadg_pml_profile prof{};
  bool kappa = false;
  wadg_pml_scheme scheme = WADG_PML_WAA;

  std::vector<int64_t> perm, iperm;  // internal -> user, user -> internal
  int64_t K0 = 0, K1 = 0;

  // device
  DevPtr q[2], rq, p, rp, geo, geof, fnrm, mat, nbr, code, sig, kap, ops, tabs, verts;
  DevPtr src, srcw, pr_elem, pr_ell, pr_out, obj, tdev, stepdev, flag, tcops, errflag;
  DevPtr stored;     // stored-matrix scheme: per PML element operators
  DevPtr dperm;      // internal -> caller element id (int32), device state exchange
  // caller-owned device memory holding the state buffers (wadg_bind_state)
  void* bound = nullptr;
  size_t bound_bytes = 0;
  // bytes this context copied between host and device memory
  size_t h2d = 0, d2h = 0;
  Budget budget;     // device-memory cap (wadg_set_memory_limit)
  bool tc = false;   // tensor-core stage kernels (TF32 or BF16 operands)
  bool bf16 = false; // BF16 operands
  // Readiness of the device side.  ready: the per-element tables and the
  // state buffers match the host mesh (the last rebuild completed).  src_ok,
  // probes_ok: the source and probe tables match the current element order
  // (the last upload of each completed).  A set-up call that fails part-way
  // clears its flag, and every call that launches kernels or touches the
  // state refuses (ESTATE) until the failed call has been repeated
  // successfully, so no kernel ever sees a freed or half-built table.
  bool ready = false;
  bool src_ok = true, probes_ok = true;
  bool ops_ok = true;   // the reference-operator tables match ref
  // quadrature class of the PML kernels (quad_capacity): 0 for the default
  // conical-product rule, 1 for a compact caller rule (wadg_set_quadrature)
  int qc = 0;
  int cur = 0;
  int nsrc = 0, nprobe = 0;
  std::vector<wadg_dipole> src_user;
  std::vector<double> probe_user;
  double t = 0.0;

  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  double graph_dt = 0.0;
  bool graph_valid = false;
  uint64_t gen = 0;   // advanced whenever the graphs are invalidated (every set-up change)
};

namespace {

wadg_status fail(wadg_ctx* c, wadg_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf; else g_err = buf;
  return s;
}

#define CK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? WADG_ENOMEM : WADG_ECUDA,      \
                  "%s: %s", #call, cudaGetErrorString(e_));                             \
  } while (0)

void dfree(DevPtr& d) {
  if (d.p && !d.borrowed) cudaFree(d.p);
  if (d.p && d.owner) d.owner->held -= d.bytes;
  d.p = nullptr;
  d.bytes = 0;
  d.owner = nullptr;
  d.borrowed = false;
}

// Every device buffer ends with kSlack spare bytes: the tensor-core kernels
// stage element blocks as bulk copies of their 16-byte-aligned cover, whose
// end may pass a buffer's last value by up to 8 bytes.
constexpr size_t kSlack = 64;

// A request beyond the active budget's cap fails as the device would when out
// of memory, before any device call.
cudaError_t dalloc(DevPtr& d, size_t bytes) {
  dfree(d);
  if (bytes == 0) return cudaSuccess;
  Budget* b = t_budget;
  if (b && b->limit && b->held + bytes > b->limit) return cudaErrorMemoryAllocation;
  cudaError_t e = cudaMalloc(&d.p, bytes + kSlack);
  if (e == cudaSuccess) {
    d.bytes = bytes;
    d.owner = b;
    if (b) b->held += bytes;
  } else {
    d.p = nullptr;
  }
  return e;
}

void invalidate_graphs(wadg_ctx* c) {
  for (auto& g : c->graph)
    if (g) { cudaGraphExecDestroy(g); g = nullptr; }
  c->graph_valid = false;
  ++c->gen;
}

// barycentric coordinates of x in user element k (lambda[4])
void barycentric(const wadg_ctx* c, int64_t k, const double* x, double* lam) {
  const double* v[4];
  for (int a = 0; a < 4; ++a) v[a] = &c->vxyz[3 * c->etov[4 * k + a]];
  double A[3][3], bvec[3];
  for (int d = 0; d < 3; ++d) {
    A[d][0] = v[1][d] - v[0][d];
    A[d][1] = v[2][d] - v[0][d];
    A[d][2] = v[3][d] - v[0][d];
    bvec[d] = x[d] - v[0][d];
  }
  double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
               A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
               A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
  double sol[3];
  for (int j = 0; j < 3; ++j) {  // Cramer's rule
    double M[3][3];
    for (int r = 0; r < 3; ++r)
      for (int cc = 0; cc < 3; ++cc) M[r][cc] = (cc == j) ? bvec[r] : A[r][cc];
    sol[j] = (M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
              M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
              M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0])) / det;
  }
  lam[1] = sol[0]; lam[2] = sol[1]; lam[3] = sol[2];
  lam[0] = 1.0 - sol[0] - sol[1] - sol[2];
}

int64_t locate(const wadg_ctx* c, const double* x, double* rst) {
  for (int64_t k = 0; k < c->K; ++k) {
    double lam[4];
    barycentric(c, k, x, lam);
    if (lam[0] >= -1e-12 && lam[1] >= -1e-12 && lam[2] >= -1e-12 && lam[3] >= -1e-12) {
      rst[0] = -1.0 + 2.0 * lam[1];
      rst[1] = -1.0 + 2.0 * lam[2];
      rst[2] = -1.0 + 2.0 * lam[3];
      return k;
    }
  }
  return -1;
}

uint64_t spread3(uint64_t x) {  // 21 bits -> every third bit
  x &= 0x1fffff;
  x = (x | x << 32) & 0x1f00000000ffffULL;
  x = (x | x << 16) & 0x1f0000ff0000ffULL;
  x = (x | x << 8) & 0x100f00f00f00f00fULL;
  x = (x | x << 4) & 0x10c30c30c30c30c3ULL;
  x = (x | x << 2) & 0x1249249249249249ULL;
  return x;
}

template <typename Real>
std::vector<Real> cvt(const std::vector<double>& a) {
  return std::vector<Real>(a.begin(), a.end());
}

template <typename Real>
wadg_status upload_ops(wadg_ctx* ctx) {
  const RefOps& R = ctx->ref;
  const int Np = R.Np, Nfp = R.Nfp, Nq = R.Nq, NF = 4 * Nfp;
  // padded, transposed layouts: DrT, DsT, DtT [Np][NpP], LIFTT [NF][NpP],
  // VqT [Np][NqP], PqT [Nq][NpP] (zeros in the padding), then the adjoint's
  const int NpP = (Np + 3) & ~3, NqP = (Nq + 3) & ~3;
  std::vector<double> h;
  for (const std::vector<double>* D : {&R.Dr, &R.Ds, &R.Dt})
    for (int j = 0; j < Np; ++j)
      for (int i = 0; i < NpP; ++i) h.push_back(i < Np ? (*D)[i * Np + j] : 0.0);
  for (int fm = 0; fm < NF; ++fm)
    for (int i = 0; i < NpP; ++i) h.push_back(i < Np ? R.LIFT[(size_t)i * NF + fm] : 0.0);
  for (int j = 0; j < Np; ++j)
    for (int q = 0; q < NqP; ++q) h.push_back(q < Nq ? R.Vq[(size_t)q * Np + j] : 0.0);
  for (int q = 0; q < Nq; ++q)
    for (int i = 0; i < NpP; ++i) h.push_back(i < Np ? R.Pq[(size_t)i * Nq + q] : 0.0);
  // for the adjoint, the same operators laid out so that consecutive threads
  // read consecutive entries: Dr, Ds, Dt [Np][NpP] (row j of D), LIFT
  // [Np][NFP] (row i), P_q [Np][NqP] (row i), V_q [Nq][NpP] (row q)
  const int NFP = (NF + 3) & ~3;
  for (const std::vector<double>* D : {&R.Dr, &R.Ds, &R.Dt})
    for (int j = 0; j < Np; ++j)
      for (int i = 0; i < NpP; ++i) h.push_back(i < Np ? (*D)[j * Np + i] : 0.0);
  for (int i = 0; i < Np; ++i)
    for (int fm = 0; fm < NFP; ++fm) h.push_back(fm < NF ? R.LIFT[(size_t)i * NF + fm] : 0.0);
  for (int i = 0; i < Np; ++i)
    for (int q = 0; q < NqP; ++q) h.push_back(q < Nq ? R.Pq[(size_t)i * Nq + q] : 0.0);
  for (int q = 0; q < Nq; ++q)
    for (int j = 0; j < NpP; ++j) h.push_back(j < Np ? R.Vq[(size_t)q * Np + j] : 0.0);
  std::vector<Real> hr = cvt<Real>(h);
  CK(dalloc(ctx->ops, hr.size() * sizeof(Real)));
  CK(cudaMemcpy(ctx->ops.p, hr.data(), hr.size() * sizeof(Real), cudaMemcpyHostToDevice));
  // Fmask [NF] | fperm [4][24][Nfp] (neighbour volume node) | fmap (neighbour face node)
  std::vector<unsigned char> t(NF + 2 * 4 * 24 * Nfp);
  for (int i = 0; i < NF; ++i) t[i] = (unsigned char)R.Fmask[i];
  for (int i = 0; i < 4 * 24 * Nfp; ++i) t[NF + i] = (unsigned char)std::max(R.fperm[i], 0);
  for (int i = 0; i < 4 * 24 * Nfp; ++i) t[NF + 4 * 24 * Nfp + i] = (unsigned char)R.fmap[i];
  CK(dalloc(ctx->tabs, t.size()));
  CK(cudaMemcpy(ctx->tabs.p, t.data(), t.size(), cudaMemcpyHostToDevice));
  if (ctx->tc) {
    // row-major Dr | Ds | Dt [Np][Np], LIFT [Np][NF], Vq [Nq][Np], Pq [Np][Nq],
    // rounded to TF32 (nearest, ties away from zero); a BF16 context rounds
    // the FP32 values once more on the device
    std::vector<float> tf;
    const bool bf = ctx->bf16;
    auto push = [&](double v) {
      float f = (float)v;
      if (!bf) {
        uint32_t u;
        std::memcpy(&u, &f, 4);
        u = (u + 0x1000u) & 0xFFFFE000u;
        std::memcpy(&f, &u, 4);
      }
      tf.push_back(f);
    };
    for (const std::vector<double>* D : {&R.Dr, &R.Ds, &R.Dt})
      for (double v : *D) push(v);
    for (double v : R.LIFT) push(v);
    for (double v : R.Vq) push(v);
    for (double v : R.Pq) push(v);
    CK(dalloc(ctx->tcops, tf.size() * 4));
    CK(cudaMemcpy(ctx->tcops.p, tf.data(), tf.size() * 4, cudaMemcpyHostToDevice));
  }
  return WADG_OK;
}

// Stored-matrix scheme (eqs. 10-13, kappa = 1): per PML element and axis the
// operators M_k^-1 M_k^{alpha} = P_h diag(alpha(x_h)) V_h, alpha = b_u, c_u,
// d_u, by a Stroud rule with N + 6 points per direction (exact to degree
// 2N + 11; the Jacobian cancels).  Built on the device in double precision.
template <typename Real>
wadg_status build_stored_ops(wadg_ctx* ctx, const double* dprof) {
  const RefOps& R = ctx->ref;
  const int Np = R.Np, NpP = (Np + 3) & ~3;
  std::vector<double> r, s_, t, w;
  stroud_rule(R.N + 6, r, s_, t, w);
  const int Nh = static_cast<int>(r.size());
  std::vector<double> rh(3 * (size_t)Nh), Vh((size_t)Nh * Np), Ph((size_t)Np * Nh);
  for (int h = 0; h < Nh; ++h) {
    rh[3 * h] = r[h];
    rh[3 * h + 1] = s_[h];
    rh[3 * h + 2] = t[h];
    std::vector<double> l = R.lagrange_at(r[h], s_[h], t[h]);
    for (int j = 0; j < Np; ++j) Vh[(size_t)h * Np + j] = l[j];
  }
  for (int i = 0; i < Np; ++i)
    for (int h = 0; h < Nh; ++h) {
      double a = 0.0;
      for (int j = 0; j < Np; ++j) a += R.Minv[i * Np + j] * Vh[(size_t)h * Np + j];
      Ph[(size_t)i * Nh + h] = a * w[h];
    }
  DevPtr drh, dVh, dPh;
  CK(dalloc(drh, rh.size() * 8));
  CK(dalloc(dVh, Vh.size() * 8));
  CK(dalloc(dPh, Ph.size() * 8));
  CK(cudaMemcpy(drh.p, rh.data(), rh.size() * 8, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(dVh.p, Vh.data(), Vh.size() * 8, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(dPh.p, Ph.data(), Ph.size() * 8, cudaMemcpyHostToDevice));
  // 3 operators per axis with kappa = 1 (B, C, D), 5 otherwise (+ K, A^-1)
  const int NB = ctx->kappa ? 5 : 3;
  const size_t bytes = (size_t)ctx->K1 * 3 * NB * Np * NpP * sizeof(Real);
  DevPtr dbad;
  CK(dalloc(ctx->stored, bytes));
  CK(dalloc(dbad, sizeof(int)));
  CK(cudaMemsetAsync(ctx->stored.p, 0, bytes, ctx->stream));
  CK(cudaMemsetAsync(dbad.p, 0, sizeof(int), ctx->stream));
  CK((launch_stored_ops<Real>(R.N, (int)ctx->K1, (int)ctx->K0, (const double*)ctx->verts.p, dprof,
                              (const double*)drh.p, (const double*)dPh.p, (const double*)dVh.p,
                              Nh, ctx->kappa, (Real*)ctx->stored.p, (int*)dbad.p, ctx->stream)));
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, dbad.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  dfree(drh);
  dfree(dVh);
  dfree(dPh);
  dfree(dbad);
  if (bad) return fail(ctx, WADG_EINVAL, "an a_u operator of the stored scheme is singular");
  return WADG_OK;
}

// The five state buffers (q[0], q[1], rq, p, rp), each followed by kSlack
// spare bytes and starting on a 256-byte boundary.
size_t state_layout(size_t qbytes, size_t pbytes, size_t off[5]) {
  const size_t sz[5] = {qbytes, qbytes, qbytes, pbytes, pbytes};
  size_t o = 0;
  for (int i = 0; i < 5; ++i) {
    off[i] = o;
    o += (sz[i] + kSlack + 255) & ~size_t(255);
  }
  return o;
}

DevPtr* state_buf(wadg_ctx* ctx, int i) {
  DevPtr* b[5] = {&ctx->q[0], &ctx->q[1], &ctx->rq, &ctx->p, &ctx->rp};
  return b[i];
}

// (re)allocate the state buffers: in the caller's bound memory when bound
// (EINVAL if it is too small), else in the library's own
wadg_status alloc_state_buffers(wadg_ctx* ctx, size_t qbytes, size_t pbytes) {
  size_t off[5];
  const size_t need = state_layout(qbytes, pbytes, off);
  const size_t sz[5] = {qbytes, qbytes, qbytes, pbytes, pbytes};
  for (int i = 0; i < 5; ++i) dfree(*state_buf(ctx, i));
  if (ctx->bound) {
    if (ctx->bound_bytes < need)
      return fail(ctx, WADG_EINVAL, "the bound state memory holds %zu bytes, the state needs %zu",
                  ctx->bound_bytes, need);
    for (int i = 0; i < 5; ++i) {
      DevPtr* d = state_buf(ctx, i);
      if (sz[i] == 0) continue;
      d->p = static_cast<unsigned char*>(ctx->bound) + off[i];
      d->bytes = sz[i];
      d->borrowed = true;
    }
    return WADG_OK;
  }
  for (int i = 0; i < 5; ++i) CK(dalloc(*state_buf(ctx, i), sz[i]));
  return WADG_OK;
}

template <typename Real>
wadg_status rebuild_typed(wadg_ctx* ctx) {
  const int64_t K = ctx->K;
  const int Np = ctx->ref.Np, Nq = ctx->ref.Nq;
  invalidate_graphs(ctx);
  // ---- classing: an element is in the PML when a vertex lies beyond u0 on
  // an active axis
  std::vector<char> is_pml(K, 0);
  if (ctx->has_prof) {
    for (int64_t k = 0; k < K; ++k)
      for (int a = 0; a < 4 && !is_pml[k]; ++a)
        for (int u = 0; u < 3; ++u) {
          bool active = ctx->prof.sigma_max[u] > 0.0 || ctx->prof.kappa_max[u] != 1.0;
          double x = ctx->vxyz[3 * ctx->etov[4 * k + a] + u];
          if (active && std::fabs(x) > ctx->prof.u0[u]) { is_pml[k] = 1; break; }
        }
  }
  // ---- order: class, then Morton code of the centroid
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t i = 0; i < ctx->nv; ++i)
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], ctx->vxyz[3 * i + d]);
      hi[d] = std::max(hi[d], ctx->vxyz[3 * i + d]);
    }
  std::vector<uint64_t> key(K);
  for (int64_t k = 0; k < K; ++k) {
    uint64_t m = 0;
    for (int d = 0; d < 3; ++d) {
      double cnt = 0.0;
      for (int a = 0; a < 4; ++a) cnt += 0.25 * ctx->vxyz[3 * ctx->etov[4 * k + a] + d];
      double s = (hi[d] > lo[d]) ? (cnt - lo[d]) / (hi[d] - lo[d]) : 0.0;
      uint64_t qd = (uint64_t)std::min(2097151.0, std::max(0.0, s * 2097151.0));
      m |= spread3(qd) << d;
    }
    key[k] = m;
  }
  ctx->perm.resize(K);
  for (int64_t k = 0; k < K; ++k) ctx->perm[k] = k;
  std::stable_sort(ctx->perm.begin(), ctx->perm.end(), [&](int64_t a, int64_t b) {
    if (is_pml[a] != is_pml[b]) return is_pml[a] < is_pml[b];
    return key[a] < key[b];
  });
  ctx->iperm.resize(K);
  for (int64_t e = 0; e < K; ++e) ctx->iperm[ctx->perm[e]] = e;
  ctx->K1 = 0;
  for (int64_t k = 0; k < K; ++k) ctx->K1 += is_pml[k];
  ctx->K0 = K - ctx->K1;
  // ---- per-element arrays in internal order
  std::vector<double> geo(K * 9), verts(K * 12);
  std::vector<Real> fn(K * 16);
  std::vector<Real> mat(K * 3);
  std::vector<int> nbr(K * 4);
  std::vector<unsigned char> code(K * 4);
  for (int64_t e = 0; e < K; ++e) {
    const int64_t k = ctx->perm[e];
    for (int i = 0; i < 9; ++i) geo[e * 9 + i] = ctx->metric_u[k * 9 + i];
    {
      // unit outward normals and Fscale = sJ/J = |grad of the face coordinate|
      const double* g = &ctx->metric_u[k * 9];
      for (int f = 0; f < 4; ++f) {
        double gx, gy, gz;
        if (f == 0) { gx = -g[6]; gy = -g[7]; gz = -g[8]; }
        else if (f == 1) { gx = -g[3]; gy = -g[4]; gz = -g[5]; }
        else if (f == 2) { gx = g[0] + g[3] + g[6]; gy = g[1] + g[4] + g[7]; gz = g[2] + g[5] + g[8]; }
        else { gx = -g[0]; gy = -g[1]; gz = -g[2]; }
        const double mag = std::sqrt(gx * gx + gy * gy + gz * gz);
        fn[e * 16 + f * 4 + 0] = (Real)(gx / mag);
        fn[e * 16 + f * 4 + 1] = (Real)(gy / mag);
        fn[e * 16 + f * 4 + 2] = (Real)(gz / mag);
        fn[e * 16 + f * 4 + 3] = (Real)mag;
      }
    }
    for (int a = 0; a < 4; ++a)
      for (int d = 0; d < 3; ++d) verts[e * 12 + a * 3 + d] = ctx->vxyz[3 * ctx->etov[4 * k + a] + d];
    double er = ctx->eps_r.empty() ? 1.0 : ctx->eps_r[k];
    double mr = ctx->mu_r.empty() ? 1.0 : ctx->mu_r[k];
    mat[e * 3 + 0] = (Real)(1.0 / er);
    mat[e * 3 + 1] = (Real)(1.0 / mr);
    mat[e * 3 + 2] = (Real)std::sqrt(mr / er);
    for (int f = 0; f < 4; ++f) {
      int64_t nk = ctx->nbr_u[k * 4 + f];
      nbr[e * 4 + f] = nk < 0 ? -1 : (int)ctx->iperm[nk];
      code[e * 4 + f] = (unsigned char)(nk < 0 ? 0 : ctx->code_u[k * 4 + f]);
    }
  }
  CK(dalloc(ctx->geo, geo.size() * 8));
  CK(cudaMemcpy(ctx->geo.p, geo.data(), geo.size() * 8, cudaMemcpyHostToDevice));
  if (ctx->tc) {   // the metric in float for the row-owned tensor-core kernels
    std::vector<float> gf(geo.begin(), geo.end());
    CK(dalloc(ctx->geof, gf.size() * 4));
    CK(cudaMemcpy(ctx->geof.p, gf.data(), gf.size() * 4, cudaMemcpyHostToDevice));
  }
  CK(dalloc(ctx->fnrm, fn.size() * sizeof(Real)));
  CK(cudaMemcpy(ctx->fnrm.p, fn.data(), fn.size() * sizeof(Real), cudaMemcpyHostToDevice));
  CK(dalloc(ctx->verts, verts.size() * 8));
  CK(cudaMemcpy(ctx->verts.p, verts.data(), verts.size() * 8, cudaMemcpyHostToDevice));
  CK(dalloc(ctx->mat, mat.size() * sizeof(Real)));
  CK(cudaMemcpy(ctx->mat.p, mat.data(), mat.size() * sizeof(Real), cudaMemcpyHostToDevice));
  CK(dalloc(ctx->nbr, nbr.size() * 4));
  CK(cudaMemcpy(ctx->nbr.p, nbr.data(), nbr.size() * 4, cudaMemcpyHostToDevice));
  CK(dalloc(ctx->code, code.size()));
  CK(cudaMemcpy(ctx->code.p, code.data(), code.size(), cudaMemcpyHostToDevice));
  {  // internal -> caller element id, for the device state exchange
    std::vector<int> pm(K);
    for (int64_t e = 0; e < K; ++e) pm[e] = (int)ctx->perm[e];
    CK(dalloc(ctx->dperm, pm.size() * 4));
    CK(cudaMemcpy(ctx->dperm.p, pm.data(), pm.size() * 4, cudaMemcpyHostToDevice));
  }
  // ---- state
  const size_t qbytes = (size_t)ctx->nb * K * 6 * Np * sizeof(Real);
  const size_t pbytes = (size_t)ctx->nb * ctx->K1 * 6 * Np * sizeof(Real);
  {
    wadg_status st = alloc_state_buffers(ctx, qbytes, pbytes);
    if (st != WADG_OK) return st;
  }
  for (int i = 0; i < 5; ++i) {
    DevPtr* d = state_buf(ctx, i);
    if (d->bytes) CK(cudaMemsetAsync(d->p, 0, d->bytes, ctx->stream));
  }
  ctx->cur = 0;
  ctx->t = 0.0;
  // ---- PML samples at the quadrature nodes (double evaluation on device)
  dfree(ctx->sig);
  dfree(ctx->kap);
  if (ctx->K1 > 0) {
    std::vector<double> rq(3 * Nq);
    for (int q = 0; q < Nq; ++q) {
      rq[3 * q] = ctx->ref.rq[q];
      rq[3 * q + 1] = ctx->ref.sq[q];
      rq[3 * q + 2] = ctx->ref.tq[q];
    }
    double prof[16];
    for (int u = 0; u < 3; ++u) {
      prof[u] = ctx->prof.u0[u];
      prof[3 + u] = ctx->prof.L[u];
      prof[6 + u] = ctx->prof.sigma_max[u];
      prof[9 + u] = ctx->prof.p_sigma[u];
      prof[12 + u] = ctx->prof.kappa_max[u];
    }
    prof[15] = ctx->prof.eps0;
    DevPtr drq, dprof;
    CK(dalloc(drq, rq.size() * 8));
    CK(dalloc(dprof, sizeof prof));
    CK(cudaMemcpy(drq.p, rq.data(), rq.size() * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(dprof.p, prof, sizeof prof, cudaMemcpyHostToDevice));
    const size_t sb = (size_t)ctx->K1 * 3 * ((Nq + 3) & ~3) * sizeof(Real);
    CK(dalloc(ctx->sig, sb));
    if (ctx->kappa) CK(dalloc(ctx->kap, sb));
    CK((launch_pml_samples<Real>(Nq, (int)ctx->K1, (int)ctx->K0, (const double*)ctx->verts.p,
                                 (const double*)drq.p, (const double*)dprof.p,
                                 (Real*)ctx->sig.p, (Real*)ctx->kap.p,
                                 ctx->scheme == WADG_PML_EC, ctx->stream)));
    CK(cudaStreamSynchronize(ctx->stream));
    dfree(drq);
    if (ctx->scheme == WADG_PML_STORED) {
      wadg_status st = build_stored_ops<Real>(ctx, (const double*)dprof.p);
      if (st != WADG_OK) {
        dfree(dprof);
        return st;
      }
      dfree(ctx->sig);   // the stored operators replace the coefficient samples
      dfree(ctx->kap);
    } else {
      dfree(ctx->stored);
    }
    dfree(dprof);
  } else {
    dfree(ctx->stored);
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return WADG_OK;
}

wadg_status rebuild(wadg_ctx* ctx) {
  ctx->ready = false;
  const wadg_status s = ctx->rs == 8 ? rebuild_typed<double>(ctx) : rebuild_typed<float>(ctx);
  ctx->ready = s == WADG_OK;
  return s;
}

template <typename Real>
wadg_status upload_sources(wadg_ctx* ctx) {
  const int Np = ctx->ref.Np;
  invalidate_graphs(ctx);
  // no source counts until the new tables are complete
  ctx->nsrc = 0;
  ctx->src_ok = false;
  std::vector<SrcDev> sd;
  std::vector<Real> w;
  for (const wadg_dipole& d : ctx->src_user) {
    double rst[3];
    int64_t k = locate(ctx, d.x, rst);
    if (k < 0)
      return fail(ctx, WADG_ENOTFOUND, "source point (%g, %g, %g) is outside the mesh", d.x[0],
                  d.x[1], d.x[2]);
    std::vector<double> ell = ctx->ref.lagrange_at(rst[0], rst[1], rst[2]);
    SrcDev s{};
    s.elem = (int)ctx->iperm[k];
    s.batch = d.batch;
    for (int u = 0; u < 3; ++u) s.dir[u] = d.dir[u];
    s.t0 = d.t0;
    s.width = d.width;
    s.amp = d.amplitude;
    sd.push_back(s);
    for (int i = 0; i < Np; ++i) {  // M_k^{-1} l(r_s) = M^{-1} l / J_k
      double a = 0.0;
      for (int j = 0; j < Np; ++j) a += ctx->ref.Minv[i * Np + j] * ell[j];
      w.push_back((Real)(a / ctx->J_u[k]));
    }
  }
  CK(dalloc(ctx->src, sd.size() * sizeof(SrcDev)));
  CK(dalloc(ctx->srcw, w.size() * sizeof(Real)));
  if (!sd.empty()) {
    CK(cudaMemcpy(ctx->src.p, sd.data(), sd.size() * sizeof(SrcDev), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->srcw.p, w.data(), w.size() * sizeof(Real), cudaMemcpyHostToDevice));
  }
  ctx->nsrc = (int)sd.size();
  ctx->src_ok = true;
  return WADG_OK;
}

wadg_status upload_probes(wadg_ctx* ctx) {
  invalidate_graphs(ctx);
  // no probe counts until the new tables are complete
  ctx->nprobe = 0;
  ctx->probes_ok = false;
  const int n = (int)(ctx->probe_user.size() / 3);
  std::vector<int> el;
  std::vector<double> ell;
  for (int i = 0; i < n; ++i) {
    double rst[3];
    int64_t k = locate(ctx, &ctx->probe_user[3 * i], rst);
    if (k < 0)
      return fail(ctx, WADG_ENOTFOUND, "probe point %d is outside the mesh", i);
    el.push_back((int)ctx->iperm[k]);
    std::vector<double> l = ctx->ref.lagrange_at(rst[0], rst[1], rst[2]);
    ell.insert(ell.end(), l.begin(), l.end());
  }
  CK(dalloc(ctx->pr_elem, el.size() * 4));
  CK(dalloc(ctx->pr_ell, ell.size() * 8));
  if (n) {
    CK(cudaMemcpy(ctx->pr_elem.p, el.data(), el.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->pr_ell.p, ell.data(), ell.size() * 8, cudaMemcpyHostToDevice));
  }
  ctx->nprobe = n;
  ctx->probes_ok = true;
  return WADG_OK;
}

wadg_status remap_points(wadg_ctx* ctx) {
  wadg_status s = ctx->rs == 8 ? upload_sources<double>(ctx) : upload_sources<float>(ctx);
  if (s != WADG_OK) return s;
  return upload_probes(ctx);
}

template <typename Real>
StageParams<Real> stage_params(wadg_ctx* ctx, int stage, double dt, double t, bool use_tdev,
                               bool pml) {
  StageParams<Real> P{};
  const int Np = ctx->ref.Np;
  P.qin = (const Real*)ctx->q[ctx->cur].p;
  P.qout = (Real*)ctx->q[ctx->cur ^ 1].p;
  P.resq = (Real*)ctx->rq.p;
  P.p = (Real*)ctx->p.p;
  P.resp = (Real*)ctx->rp.p;
  P.geo = (const double*)ctx->geo.p;
  P.geof = (const float*)ctx->geof.p;
  P.fnrm = (const Real*)ctx->fnrm.p;
  P.mat = (const Real*)ctx->mat.p;
  P.nbr = (const int*)ctx->nbr.p;
  P.code = (const unsigned char*)ctx->code.p;
  P.sig = (const Real*)ctx->sig.p;
  P.kap = (const Real*)ctx->kap.p;
  P.ops = (const Real*)ctx->ops.p;
  P.stored = (const Real*)ctx->stored.p;
  P.tabs = (const unsigned char*)ctx->tabs.p;
  P.strideQ = ctx->K * 6 * Np;
  P.strideP = ctx->K1 * 6 * Np;
  P.K0 = (int)ctx->K0;
  P.e_begin = pml ? (int)ctx->K0 : 0;
  P.n_elem = pml ? (int)ctx->K1 : (int)ctx->K0;
  P.nsrc = ctx->nsrc;
  P.src = (const SrcDev*)ctx->src.p;
  P.src_w = (const Real*)ctx->srcw.p;
  P.rk_a = kRkA[stage];
  P.rk_b = kRkB[stage];
  P.rk_c = kRkC.c[stage];
  P.dt = dt;
  P.t = t;
  P.t_dev = use_tdev ? (const double*)ctx->tdev.p : nullptr;
  P.eps0 = ctx->has_prof ? ctx->prof.eps0 : 1.0;
  P.alpha = 1.0;
  P.tcops = ctx->tcops.p;
  P.err = (int*)ctx->errflag.p;
  P.inject = ctx->tc ? (int*)ctx->errflag.p + 1 : nullptr;
  return P;
}

// the PML-class launch of a stage: the stored-matrix kernel, the tensor-core
// kernel (TF32 contexts) or the CUDA-core kernel
template <typename Real>
cudaError_t launch_pml_class(wadg_ctx* ctx, const StageParams<Real>& P, cudaStream_t s) {
  if (ctx->scheme == WADG_PML_STORED)
    return launch_stage_stored<Real>(ctx->N, ctx->kappa, P, ctx->nb, s);
  if constexpr (std::is_same<Real, float>::value) {
    if (ctx->tc) {
      // compact volume rules: the row-owned kernel; (N+1)^3 rules: the other
      if (ctx->qc == 1) return launch_pml_tc_rows(ctx->N, P, ctx->nb, s, ctx->bf16);
      return launch_stage_tc(ctx->N, true, P, ctx->nb, s, ctx->bf16, ctx->qc);
    }
  }
  return launch_stage<Real>(ctx->N, true, ctx->kappa, P, ctx->nb, s, ctx->qc);
}
template <typename Real>
cudaError_t launch_pml_class(wadg_ctx* ctx, const StageParams<Real>& P) {
  return launch_pml_class<Real>(ctx, P, ctx->stream);
}

// the non-PML class of a stage on stream s (the kernel of the context's kind)
template <typename Real>
cudaError_t launch_std_class(wadg_ctx* ctx, const StageParams<Real>& P, cudaStream_t s) {
  if constexpr (std::is_same<Real, float>::value)
    if (ctx->tc) return launch_stage_tc(ctx->N, false, P, ctx->nb, s, ctx->bf16, ctx->qc);
  return launch_stage<Real>(ctx->N, false, false, P, ctx->nb, s);
}

// one element class of one stage of a context, on stream s, with the device
// clock (graph replays); tile: elements per tile of the CUDA-core kernels
// (0: the largest)
cudaError_t launch_member_class(wadg_ctx* x, int st, double dt, bool pml, int tile,
                                cudaStream_t s) {
  if (x->rs == 8) {
    StageParams<double> P = stage_params<double>(x, st, dt, 0.0, true, pml);
    P.tile_elems = tile;
    return pml ? launch_pml_class<double>(x, P, s) : launch_std_class<double>(x, P, s);
  }
  StageParams<float> P = stage_params<float>(x, st, dt, 0.0, true, pml);
  P.tile_elems = x->tc ? 0 : tile;
  return pml ? launch_pml_class<float>(x, P, s) : launch_std_class<float>(x, P, s);
}

template <typename Real>
wadg_status issue_stage(wadg_ctx* ctx, int stage, double dt, double t, bool use_tdev) {
  if (ctx->tc) {
    StageParams<float> A = stage_params<float>(ctx, stage, dt, t, use_tdev, false);
    CK(launch_stage_tc(ctx->N, false, A, ctx->nb, ctx->stream, ctx->bf16, ctx->qc));
    if (ctx->K1 > 0) {
      StageParams<float> B = stage_params<float>(ctx, stage, dt, t, use_tdev, true);
      CK(launch_pml_class<float>(ctx, B));
    }
    ctx->cur ^= 1;
    return WADG_OK;
  }
  StageParams<Real> A = stage_params<Real>(ctx, stage, dt, t, use_tdev, false);
  CK(launch_stage<Real>(ctx->N, false, false, A, ctx->nb, ctx->stream));
  if (ctx->K1 > 0) {
    StageParams<Real> B = stage_params<Real>(ctx, stage, dt, t, use_tdev, true);
    CK(launch_pml_class<Real>(ctx, B));
  }
  ctx->cur ^= 1;
  return WADG_OK;
}

// one stage of a step graph with the two element classes on parallel
// branches: the PML class on the context's stream, the non-PML class on the
// branch (they write disjoint elements and read the same stage input), so
// one class's blocks take the SMs the other's leave at its tail
template <typename Real>
wadg_status issue_stage_branches(wadg_ctx* ctx, int stage, double dt) {
  CK(cudaEventRecord(ctx->ev_fork, ctx->stream));
  CK(cudaStreamWaitEvent(ctx->aux, ctx->ev_fork, 0));
  if (ctx->tc) {
    StageParams<float> B = stage_params<float>(ctx, stage, dt, 0.0, true, true);
    CK(launch_pml_class<float>(ctx, B));
    StageParams<float> A = stage_params<float>(ctx, stage, dt, 0.0, true, false);
    CK(launch_stage_tc(ctx->N, false, A, ctx->nb, ctx->aux, ctx->bf16, ctx->qc));
  } else {
    StageParams<Real> B = stage_params<Real>(ctx, stage, dt, 0.0, true, true);
    CK(launch_pml_class<Real>(ctx, B));
    StageParams<Real> A = stage_params<Real>(ctx, stage, dt, 0.0, true, false);
    CK(launch_stage<Real>(ctx->N, false, false, A, ctx->nb, ctx->aux));
  }
  CK(cudaEventRecord(ctx->ev_join, ctx->aux));
  CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0));
  ctx->cur ^= 1;
  return WADG_OK;
}

wadg_status issue_step(wadg_ctx* ctx, double dt) {
  const bool branches = ctx->K1 > 0 && ctx->K0 > 0 && ctx->aux;
  for (int s = 0; s < 5; ++s) {
    wadg_status st;
    if (branches)
      st = ctx->rs == 8 ? issue_stage_branches<double>(ctx, s, dt)
                        : issue_stage_branches<float>(ctx, s, dt);
    else
      st = ctx->rs == 8 ? issue_stage<double>(ctx, s, dt, 0.0, true)
                        : issue_stage<float>(ctx, s, dt, 0.0, true);
    if (st != WADG_OK) return st;
  }
  if (ctx->nprobe > 0) {
    ProbeParams pp{};
    pp.q = ctx->q[ctx->cur].p;
    pp.strideQ = ctx->K * 6 * ctx->ref.Np;
    pp.nprobe = ctx->nprobe;
    pp.nb = ctx->nb;
    pp.Np = ctx->ref.Np;
    pp.elem = (const int*)ctx->pr_elem.p;
    pp.ell = (const double*)ctx->pr_ell.p;
    pp.out = (double*)ctx->pr_out.p;
    pp.obj = (double*)ctx->obj.p;
    pp.step = (const int64_t*)ctx->stepdev.p;
    CK(launch_probes(ctx->rs == 8, pp, ctx->stream));
  }
  CK(launch_advance((double*)ctx->tdev.p, (int64_t*)ctx->stepdev.p, dt, ctx->stream));
  return WADG_OK;
}

wadg_status capture_graphs(wadg_ctx* ctx, double dt) {
  invalidate_graphs(ctx);
  if (ctx->K1 > 0 && ctx->K0 > 0 && !ctx->aux) {   // the branch of the two element classes
    CK(cudaStreamCreateWithFlags(&ctx->aux, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming));
  }
  const int start = ctx->cur;
  for (int g = 0; g < 2; ++g) {
    ctx->cur = g;
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    wadg_status st = issue_step(ctx, dt);
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
    if (st != WADG_OK) return st;
    CK(e);
    e = cudaGraphInstantiate(&ctx->graph[g], graph, 0);
    cudaGraphDestroy(graph);
    CK(e);
  }
  ctx->cur = start;
  ctx->graph_dt = dt;
  ctx->graph_valid = true;
  return WADG_OK;
}

// bounded device waits that gave up leave a flag behind
wadg_status check_err_flag(wadg_ctx* ctx) {
  int e = 0;
  CK(cudaMemcpyAsync(&e, ctx->errflag.p, 4, cudaMemcpyDeviceToHost, ctx->stream));
  ctx->d2h += 4;
  CK(cudaStreamSynchronize(ctx->stream));
  if (e) {
    CK(cudaMemset(ctx->errflag.p, 0, 4));
    if (e & 1)
      return fail(ctx, WADG_ETIMEOUT, "a tensor-core stage kernel gave up waiting for its products");
    return fail(ctx, WADG_ECUDA, "a device index check failed (checked build): mesh tables corrupt");
  }
  return WADG_OK;
}

wadg_status need_mesh(wadg_ctx* ctx) {
  if (!ctx) return fail(nullptr, WADG_EINVAL, "null context");
  if (!ctx->has_mesh) return fail(ctx, WADG_ESTATE, "no mesh set");
  return WADG_OK;
}

// every device table the stage, probe and state calls read is complete
wadg_status need_ready(wadg_ctx* ctx) {
  wadg_status s = need_mesh(ctx);
  if (s != WADG_OK) return s;
  if (!ctx->ops_ok)
    return fail(ctx, WADG_ESTATE, "the operator tables are incomplete after a failed call: "
                "repeat wadg_set_quadrature");
  if (!ctx->ready)
    return fail(ctx, WADG_ESTATE,
                "the device tables are incomplete after a failed set-up call: repeat "
                "wadg_set_mesh, wadg_set_materials or wadg_set_pml_profile");
  if (!ctx->src_ok)
    return fail(ctx, WADG_ESTATE, "the sources are not mapped after a failed call: repeat wadg_set_sources");
  if (!ctx->probes_ok)
    return fail(ctx, WADG_ESTATE, "the probes are not mapped after a failed call: repeat wadg_set_probes");
  return WADG_OK;
}

template <typename Real>
static wadg_status set_state_t(wadg_ctx* ctx, const double* q) {
  const int Np = ctx->ref.Np;
  const int64_t K = ctx->K;
  std::vector<Real> hq((size_t)ctx->nb * K * 6 * Np, Real(0));
  std::vector<Real> hp((size_t)ctx->nb * ctx->K1 * 6 * Np, Real(0));
  if (q) {
    for (int b = 0; b < ctx->nb; ++b)
      for (int64_t e = 0; e < K; ++e) {
        const int64_t k = ctx->perm[e];
        const double* src = q + (((size_t)b * K + k) * 12) * Np;
        Real* dq = &hq[(((size_t)b * K + e) * 6) * Np];
        for (int i = 0; i < 6 * Np; ++i) dq[i] = (Real)src[i];
        if (e >= ctx->K0) {
          Real* dp = &hp[(((size_t)b * ctx->K1 + (e - ctx->K0)) * 6) * Np];
          for (int i = 0; i < 6 * Np; ++i) dp[i] = (Real)src[6 * Np + i];
        }
      }
  }
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->cur = 0;
  if (!hq.empty())
    CK(cudaMemcpy(ctx->q[0].p, hq.data(), hq.size() * sizeof(Real), cudaMemcpyHostToDevice));
  if (!hp.empty())
    CK(cudaMemcpy(ctx->p.p, hp.data(), hp.size() * sizeof(Real), cudaMemcpyHostToDevice));
  ctx->h2d += (hq.size() + hp.size()) * sizeof(Real);
  CK(cudaMemset(ctx->rq.p, 0, ctx->rq.bytes));
  if (ctx->rp.bytes) CK(cudaMemset(ctx->rp.p, 0, ctx->rp.bytes));
  CK(cudaMemset(ctx->obj.p, 0, ctx->obj.bytes));
  return WADG_OK;
}

template <typename Real>
static wadg_status get_state_t(wadg_ctx* ctx, double* q) {
  const int Np = ctx->ref.Np;
  const int64_t K = ctx->K;
  std::vector<Real> hq((size_t)ctx->nb * K * 6 * Np);
  std::vector<Real> hp((size_t)ctx->nb * ctx->K1 * 6 * Np);
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaMemcpy(hq.data(), ctx->q[ctx->cur].p, hq.size() * sizeof(Real), cudaMemcpyDeviceToHost));
  if (!hp.empty())
    CK(cudaMemcpy(hp.data(), ctx->p.p, hp.size() * sizeof(Real), cudaMemcpyDeviceToHost));
  ctx->d2h += (hq.size() + hp.size()) * sizeof(Real);
  for (int b = 0; b < ctx->nb; ++b)
    for (int64_t e = 0; e < K; ++e) {
      const int64_t k = ctx->perm[e];
      double* dst = q + (((size_t)b * K + k) * 12) * Np;
      const Real* sq = &hq[(((size_t)b * K + e) * 6) * Np];
      for (int i = 0; i < 6 * Np; ++i) dst[i] = (double)sq[i];
      if (e >= ctx->K0) {
        const Real* sp = &hp[(((size_t)b * ctx->K1 + (e - ctx->K0)) * 6) * Np];
        for (int i = 0; i < 6 * Np; ++i) dst[6 * Np + i] = (double)sp[i];
      } else {
        for (int i = 0; i < 6 * Np; ++i) dst[6 * Np + i] = 0.0;
      }
    }
  return WADG_OK;
}

// device-resident exchange: a kernel on the context's stream converts
// between the caller's array (ABI layout, double) and the internal blocks
template <typename Real>
static wadg_status set_state_dev(wadg_ctx* ctx, const double* q) {
  ctx->cur = 0;
  if (q) {
    CK(launch_state_exchange<Real>(true, (const int*)ctx->dperm.p, ctx->K, ctx->K0, ctx->ref.Np,
                                   ctx->nb, const_cast<double*>(q), (Real*)ctx->q[0].p,
                                   (Real*)ctx->p.p, ctx->stream));
  } else {
    if (ctx->q[0].bytes) CK(cudaMemsetAsync(ctx->q[0].p, 0, ctx->q[0].bytes, ctx->stream));
    if (ctx->p.bytes) CK(cudaMemsetAsync(ctx->p.p, 0, ctx->p.bytes, ctx->stream));
  }
  CK(cudaMemsetAsync(ctx->rq.p, 0, ctx->rq.bytes, ctx->stream));
  if (ctx->rp.bytes) CK(cudaMemsetAsync(ctx->rp.p, 0, ctx->rp.bytes, ctx->stream));
  CK(cudaMemsetAsync(ctx->obj.p, 0, ctx->obj.bytes, ctx->stream));
  return WADG_OK;
}

template <typename Real>
static wadg_status get_state_dev(wadg_ctx* ctx, double* q) {
  CK(launch_state_exchange<Real>(false, (const int*)ctx->dperm.p, ctx->K, ctx->K0, ctx->ref.Np,
                                 ctx->nb, q, (Real*)ctx->q[ctx->cur].p, (Real*)ctx->p.p,
                                 ctx->stream));
  return WADG_OK;
}

// exchange through host memory: the caller's array moves as it is, in one
// copy, through a device staging buffer that the exchange kernel converts
// (instead of a per-element conversion loop on one host thread); when the
// staging buffer cannot be had (a memory cap), the host loops above convert
template <typename Real>
static wadg_status set_state_host(wadg_ctx* ctx, const double* q) {
  const size_t ub = (size_t)ctx->nb * ctx->K * 12 * ctx->ref.Np * sizeof(double);
  DevPtr st;
  if (q && dalloc(st, ub) == cudaSuccess) {
    wadg_status s = WADG_OK;
    cudaError_t e = cudaMemcpyAsync(st.p, q, ub, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) s = set_state_dev<Real>(ctx, static_cast<const double*>(st.p));
    if (e == cudaSuccess && s == WADG_OK) e = cudaStreamSynchronize(ctx->stream);
    dfree(st);
    if (e != cudaSuccess) return fail(ctx, WADG_ECUDA, "state upload: %s", cudaGetErrorString(e));
    if (s == WADG_OK) ctx->h2d += ub;
    return s;
  }
  cudaGetLastError();   // a refused allocation must not be read as a later launch's error
  return set_state_t<Real>(ctx, q);
}

template <typename Real>
static wadg_status get_state_host(wadg_ctx* ctx, double* q) {
  const size_t ub = (size_t)ctx->nb * ctx->K * 12 * ctx->ref.Np * sizeof(double);
  DevPtr st;
  if (dalloc(st, ub) == cudaSuccess) {
    wadg_status s = get_state_dev<Real>(ctx, static_cast<double*>(st.p));
    cudaError_t e = cudaSuccess;
    if (s == WADG_OK) e = cudaMemcpyAsync(q, st.p, ub, cudaMemcpyDeviceToHost, ctx->stream);
    if (s == WADG_OK && e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    dfree(st);
    if (e != cudaSuccess) return fail(ctx, WADG_ECUDA, "state download: %s", cudaGetErrorString(e));
    if (s == WADG_OK) ctx->d2h += ub;
    return s;
  }
  cudaGetLastError();   // a refused allocation must not be read as a later launch's error
  return get_state_t<Real>(ctx, q);
}

}  // namespace

extern "C" {

wadg_status wadg_create(int N, wadg_precision prec, int32_t n_batch, int device,
                        void* cuda_stream, wadg_ctx** out) {
  wadg_ctx* ctx = nullptr;
  if (!out) return fail(nullptr, WADG_EINVAL, "out is NULL");
  *out = nullptr;
  if (N < 1 || N > 5) return fail(nullptr, WADG_EINVAL, "N must be in 1..5 (got %d)", N);
  if (prec != WADG_FP64 && prec != WADG_FP32 && prec != WADG_TF32 && prec != WADG_BF16)
    return fail(nullptr, WADG_EINVAL, "unknown precision %d", prec);
  if ((prec == WADG_TF32 || prec == WADG_BF16) && !tc_supported(N, false, prec == WADG_BF16, 1))
    return fail(nullptr, WADG_EUNSUPPORTED, "the tensor-core stage is built for N <= 5");
  if (n_batch < 1) return fail(nullptr, WADG_EINVAL, "n_batch must be >= 1");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return fail(nullptr, WADG_ECUDA, "CUDA device %d not available", device);
  if (cudaSetDevice(device) != cudaSuccess)
    return fail(nullptr, WADG_ECUDA, "cudaSetDevice(%d) failed", device);
  ctx = new wadg_ctx();
  BudgetScope budget_scope(&ctx->budget);
  ctx->N = N;
  ctx->prec = prec;
  ctx->nb = n_batch;
  ctx->device = device;
  ctx->rs = prec == WADG_FP64 ? 8 : 4;
  ctx->tc = prec == WADG_TF32 || prec == WADG_BF16;
  ctx->bf16 = prec == WADG_BF16;
  const char* e = nullptr;
  if (!build_ref_ops(N, ctx->ref, &e)) {
    delete ctx;
    return fail(nullptr, WADG_EINVAL, "%s", e);
  }
  if (cuda_stream) {
    ctx->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete ctx;
      return fail(nullptr, WADG_ECUDA, "cannot create a stream");
    }
    ctx->own_stream = true;
  }
  wadg_status s = ctx->rs == 8 ? upload_ops<double>(ctx) : upload_ops<float>(ctx);
  if (s == WADG_OK) {
    cudaError_t ce = ctx->rs == 8 ? configure_stage_kernels<double>(N)
                                  : configure_stage_kernels<float>(N);
    if (ce == cudaSuccess && ctx->tc) ce = configure_tc_kernels(N, ctx->bf16);
    if (ce == cudaSuccess && ctx->tc) ce = configure_tc_rows(N, ctx->bf16);
    if (ce == cudaSuccess)
      ce = ctx->rs == 8 ? configure_stored_kernels<double>(N) : configure_stored_kernels<float>(N);
    if (ce == cudaSuccess && !ctx->tc)
      ce = ctx->rs == 8 ? configure_adjoint_kernels<double>(N) : configure_adjoint_kernels<float>(N);
    if (ce != cudaSuccess) s = fail(ctx, WADG_ECUDA, "kernel set-up: %s", cudaGetErrorString(ce));
  }
  if (s == WADG_OK) {
    cudaError_t ce = cudaSuccess;
    if (ce == cudaSuccess) ce = dalloc(ctx->tdev, 8);
    if (ce == cudaSuccess) ce = dalloc(ctx->stepdev, 8);
    if (ce == cudaSuccess) ce = dalloc(ctx->flag, 4);
    // [0] error flag of the bounded waits, [1] armed failure-detection request
    if (ce == cudaSuccess) ce = dalloc(ctx->errflag, 8);
    if (ce == cudaSuccess) ce = cudaMemset(ctx->errflag.p, 0, 8);
    if (ce == cudaSuccess) ce = dalloc(ctx->obj, 8 * (size_t)n_batch);
    if (ce == cudaSuccess) ce = cudaMemset(ctx->obj.p, 0, 8 * (size_t)n_batch);
    if (ce != cudaSuccess) s = fail(nullptr, WADG_ECUDA, "%s", cudaGetErrorString(ce));
  } else {
    g_err = ctx->err;
  }
  if (s != WADG_OK) {
    wadg_destroy(ctx);
    return s;
  }
  *out = ctx;
  return WADG_OK;
}

wadg_status wadg_destroy(wadg_ctx* ctx) {
  if (!ctx) return WADG_OK;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  invalidate_graphs(ctx);
  for (DevPtr* d : {&ctx->q[0], &ctx->q[1], &ctx->rq, &ctx->p, &ctx->rp, &ctx->geo, &ctx->geof, &ctx->fnrm, &ctx->mat,
                    &ctx->nbr, &ctx->code, &ctx->sig, &ctx->kap, &ctx->ops, &ctx->tabs,
                    &ctx->verts, &ctx->src, &ctx->srcw, &ctx->pr_elem, &ctx->pr_ell,
                    &ctx->pr_out, &ctx->obj, &ctx->tdev, &ctx->stepdev, &ctx->flag,
                    &ctx->tcops, &ctx->errflag, &ctx->stored, &ctx->dperm})
    dfree(*d);
  if (ctx->aux) cudaStreamDestroy(ctx->aux);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return WADG_OK;
}

wadg_status wadg_set_mesh(wadg_ctx* ctx, int64_t nv, const double* vxyz, int64_t K,
                          const int64_t* etov) {
  return wadg_set_mesh_periodic(ctx, nv, vxyz, K, etov, nullptr);
}

wadg_status wadg_set_mesh_periodic(wadg_ctx* ctx, int64_t nv, const double* vxyz, int64_t K,
                                   const int64_t* etov, const int64_t* vcanon) {
  if (!ctx) return fail(nullptr, WADG_EINVAL, "null context");
  if (nv < 4 || K < 1 || !vxyz || !etov) return fail(ctx, WADG_EINVAL, "empty mesh");
  if (K > (int64_t)1 << 30) return fail(ctx, WADG_EINVAL, "too many elements");
  cudaSetDevice(ctx->device);
  BudgetScope budget_scope(&ctx->budget);
  for (int64_t i = 0; i < 4 * K; ++i)
    if (etov[i] < 0 || etov[i] >= nv)
      return fail(ctx, WADG_EINVAL, "etov[%lld] = %lld out of range", (long long)i,
                  (long long)etov[i]);
  if (vcanon)
    for (int64_t i = 0; i < nv; ++i)
      if (vcanon[i] < 0 || vcanon[i] >= nv)
        return fail(ctx, WADG_EINVAL, "vcanon[%lld] = %lld out of range", (long long)i,
                    (long long)vcanon[i]);
  // face keys use the periodic representatives of the vertices
  auto cv = [vcanon](int64_t v) { return vcanon ? vcanon[v] : v; };
  ctx->has_mesh = false;
  ctx->ready = false;
  // the point tables refer to the old element order: drop them
  invalidate_graphs(ctx);
  for (DevPtr* d : {&ctx->src, &ctx->srcw, &ctx->pr_elem, &ctx->pr_ell}) dfree(*d);
  ctx->nsrc = ctx->nprobe = 0;
  ctx->src_ok = ctx->probes_ok = true;
  ctx->K = K;
  ctx->nv = nv;
  ctx->vxyz.assign(vxyz, vxyz + 3 * nv);
  ctx->etov.assign(etov, etov + 4 * K);
  ctx->eps_r.clear();
  ctx->mu_r.clear();
  ctx->has_prof = false;
  ctx->kappa = false;
  ctx->src_user.clear();
  ctx->probe_user.clear();
  // ---- affine geometry in double
  ctx->metric_u.assign(9 * K, 0.0);
  ctx->J_u.assign(K, 0.0);
  ctx->fscale_max = 0.0;
  for (int64_t k = 0; k < K; ++k) {
    const double* v[4];
    for (int a = 0; a < 4; ++a) v[a] = &vxyz[3 * etov[4 * k + a]];
    double A[3][3];  // columns dx/dr, dx/ds, dx/dt
    for (int d = 0; d < 3; ++d) {
      A[d][0] = 0.5 * (v[1][d] - v[0][d]);
      A[d][1] = 0.5 * (v[2][d] - v[0][d]);
      A[d][2] = 0.5 * (v[3][d] - v[0][d]);
    }
    double c00 = A[1][1] * A[2][2] - A[1][2] * A[2][1];
    double c01 = A[1][2] * A[2][0] - A[1][0] * A[2][2];
    double c02 = A[1][0] * A[2][1] - A[1][1] * A[2][0];
    double J = A[0][0] * c00 + A[0][1] * c01 + A[0][2] * c02;
    if (!(J > 0.0))
      return fail(ctx, WADG_EINVAL, "element %lld has non-positive Jacobian %g", (long long)k, J);
    double inv[3][3];  // inverse: rows grad r, grad s, grad t
    inv[0][0] = c00 / J;
    inv[1][0] = c01 / J;
    inv[2][0] = c02 / J;
    inv[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / J;
    inv[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / J;
    inv[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) / J;
    inv[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / J;
    inv[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) / J;
    inv[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / J;
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) ctx->metric_u[9 * k + 3 * r + c] = inv[r][c];
    ctx->J_u[k] = J;
    double g[4][3];
    for (int d = 0; d < 3; ++d) {
      g[0][d] = -inv[2][d];
      g[1][d] = -inv[1][d];
      g[2][d] = inv[0][d] + inv[1][d] + inv[2][d];
      g[3][d] = -inv[0][d];
    }
    for (int f = 0; f < 4; ++f)
      ctx->fscale_max = std::max(
          ctx->fscale_max, std::sqrt(g[f][0] * g[f][0] + g[f][1] * g[f][1] + g[f][2] * g[f][2]));
  }
  // ---- face connectivity by sorted vertex triples
  struct FaceKey {
    int64_t a, b, c, id;
  };
  std::vector<FaceKey> fk(4 * K);
  for (int64_t k = 0; k < K; ++k)
    for (int f = 0; f < 4; ++f) {
      int64_t v3[3];
      for (int i = 0; i < 3; ++i) v3[i] = cv(etov[4 * k + kFaceVerts[f][i]]);
      std::sort(v3, v3 + 3);
      fk[4 * k + f] = {v3[0], v3[1], v3[2], 4 * k + f};
    }
  std::sort(fk.begin(), fk.end(), [](const FaceKey& x, const FaceKey& y) {
    if (x.a != y.a) return x.a < y.a;
    if (x.b != y.b) return x.b < y.b;
    if (x.c != y.c) return x.c < y.c;
    return x.id < y.id;
  });
  ctx->nbr_u.assign(4 * K, -1);
  ctx->code_u.assign(4 * K, 0);
  auto same = [](const FaceKey& x, const FaceKey& y) { return x.a == y.a && x.b == y.b && x.c == y.c; };
  for (size_t i = 0; i < fk.size();) {
    size_t j = i + 1;
    while (j < fk.size() && same(fk[i], fk[j])) ++j;
    if (j - i > 2)
      return fail(ctx, WADG_EINVAL, "face (%lld,%lld,%lld) shared by %d elements",
                  (long long)fk[i].a, (long long)fk[i].b, (long long)fk[i].c, (int)(j - i));
    if (j - i == 2) {
      for (int side = 0; side < 2; ++side) {
        int64_t me = fk[i + side].id, ot = fk[i + 1 - side].id;
        int64_t k = me / 4, f = me % 4, k2 = ot / 4, f2 = ot % 4;
        int64_t gv[3], hv[3];
        for (int a = 0; a < 3; ++a) {
          gv[a] = cv(etov[4 * k + kFaceVerts[f][a]]);
          hv[a] = cv(etov[4 * k2 + kFaceVerts[f2][a]]);
        }
        int rot = -1;
        for (int r = 0; r < 6 && rot < 0; ++r)
          if (hv[0] == gv[kFacePerm[r][0]] && hv[1] == gv[kFacePerm[r][1]] &&
              hv[2] == gv[kFacePerm[r][2]])
            rot = r;
        if (rot < 0) return fail(ctx, WADG_EINVAL, "degenerate face in element %lld", (long long)k);
        ctx->nbr_u[me] = k2;
        ctx->code_u[me] = (int)(f2 * 6 + rot);
      }
    }
    i = j;
  }
  ctx->has_mesh = true;
  return rebuild(ctx);
}

wadg_status wadg_set_materials(wadg_ctx* ctx, const double* eps_r, const double* mu_r) {
  wadg_status s = need_mesh(ctx);
  if (s != WADG_OK) return s;
  cudaSetDevice(ctx->device);
  BudgetScope budget_scope(&ctx->budget);
  for (int64_t k = 0; k < ctx->K; ++k)
    if ((eps_r && !(eps_r[k] > 0)) || (mu_r && !(mu_r[k] > 0)))
      return fail(ctx, WADG_EINVAL, "material of element %lld not positive", (long long)k);
  if (eps_r) ctx->eps_r.assign(eps_r, eps_r + ctx->K); else ctx->eps_r.clear();
  if (mu_r) ctx->mu_r.assign(mu_r, mu_r + ctx->K); else ctx->mu_r.clear();
  s = rebuild(ctx);
  if (s != WADG_OK) return s;
  return remap_points(ctx);
}

wadg_status wadg_set_pml_profile(wadg_ctx* ctx, const wadg_pml_profile* prof,
                                 wadg_pml_scheme scheme) {
  wadg_status s = need_mesh(ctx);
  if (s != WADG_OK) return s;
  cudaSetDevice(ctx->device);
  BudgetScope budget_scope(&ctx->budget);
  if (scheme != WADG_PML_WAA && scheme != WADG_PML_STORED && scheme != WADG_PML_EC)
    return fail(ctx, WADG_EINVAL, "unknown PML scheme %d", (int)scheme);
  if (prof) {
    for (int u = 0; u < 3; ++u) {
      if (!(prof->L[u] > 0) || prof->sigma_max[u] < 0 || !(prof->kappa_max[u] >= 1.0) ||
          !(prof->p_sigma[u] >= 0))
        return fail(ctx, WADG_EINVAL, "bad PML profile on axis %d", u);
    }
    if (!(prof->eps0 > 0)) return fail(ctx, WADG_EINVAL, "eps0 must be positive");
    bool kap = false;
    for (int u = 0; u < 3; ++u)
      if (prof->kappa_max[u] != 1.0) kap = true;
    if (kap && ctx->tc && scheme != WADG_PML_STORED)
      return fail(ctx, WADG_EUNSUPPORTED, "kappa_max != 1 is not built for the tensor-core stage");
    if (ctx->tc && scheme != WADG_PML_STORED && !tc_supported(ctx->N, false, ctx->bf16, ctx->qc))
      return fail(ctx, WADG_EUNSUPPORTED,
                  "TF32 operands at N = 5 need a compact volume rule (wadg_set_quadrature)");
    ctx->has_prof = true;
    ctx->prof = *prof;
    ctx->kappa = kap;
    ctx->scheme = scheme;
  } else {
    ctx->has_prof = false;
    ctx->kappa = false;
    ctx->scheme = WADG_PML_WAA;
  }
  s = rebuild(ctx);
  if (s != WADG_OK) return s;
  return remap_points(ctx);
}

wadg_status wadg_set_quadrature(wadg_ctx* ctx, int32_t nq, const double* rstw) {
  if (!ctx) return fail(nullptr, WADG_EINVAL, "null context");
  cudaSetDevice(ctx->device);
  BudgetScope budget_scope(&ctx->budget);
  const int N = ctx->N;
  std::vector<double> r, s_, t, w;
  int qc = 0, cap = 0;
  if (rstw) {
    if (nq < 1) return fail(ctx, WADG_EINVAL, "empty quadrature rule");
    if (nq <= compact_nq(N)) qc = 1;
    else if (nq <= quad_capacity(N, 0)) qc = 0;
    else
      return fail(ctx, WADG_EUNSUPPORTED, "the PML kernels hold at most %d volume quadrature "
                  "points at N = %d (got %d)", quad_capacity(N, 0), N, (int)nq);
    cap = quad_capacity(N, qc);
    for (int q = 0; q < nq; ++q) {
      r.push_back(rstw[4 * q]);
      s_.push_back(rstw[4 * q + 1]);
      t.push_back(rstw[4 * q + 2]);
      w.push_back(rstw[4 * q + 3]);
    }
  } else {
    stroud_rule(N + 1, r, s_, t, w);
    cap = quad_capacity(N, 0);
  }
  if (ctx->tc && ctx->has_prof && ctx->scheme != WADG_PML_STORED &&
      !tc_supported(N, false, ctx->bf16, qc))
    return fail(ctx, WADG_EUNSUPPORTED,
                "TF32 operands at N = 5 need a compact volume rule with the PML set");
  RefOps R = ctx->ref;
  const char* e = nullptr;
  if (!set_volume_rule(R, r, s_, t, w, cap, &e)) return fail(ctx, WADG_EINVAL, "%s", e);
  // the operator tables and (with a mesh) every per-element table follow
  ctx->ready = false;
  invalidate_graphs(ctx);
  ctx->ref = R;
  ctx->qc = qc;
  ctx->ops_ok = false;
  wadg_status st = ctx->rs == 8 ? upload_ops<double>(ctx) : upload_ops<float>(ctx);
  if (st != WADG_OK) return st;
  ctx->ops_ok = true;
  if (!ctx->has_mesh) return WADG_OK;
  st = rebuild(ctx);
  if (st != WADG_OK) return st;
  return remap_points(ctx);
}

wadg_status wadg_set_sources(wadg_ctx* ctx, int32_t n, const wadg_dipole* src) {
  wadg_status s = need_mesh(ctx);
  if (s != WADG_OK) return s;
  cudaSetDevice(ctx->device);
  BudgetScope budget_scope(&ctx->budget);
  if (n < 0 || (n > 0 && !src)) return fail(ctx, WADG_EINVAL, "bad source list");
  for (int i = 0; i < n; ++i) {
    if (src[i].batch < 0 || src[i].batch >= ctx->nb)
      return fail(ctx, WADG_EINVAL, "source %d: batch %d out of range", i, src[i].batch);
    if (!(src[i].width > 0)) return fail(ctx, WADG_EINVAL, "source %d: width must be > 0", i);
  }
  ctx->src_user.assign(src, src + n);
  return ctx->rs == 8 ? upload_sources<double>(ctx) : upload_sources<float>(ctx);
}

wadg_status wadg_set_probes(wadg_ctx* ctx, int32_t n, const double* xyz) {
  wadg_status s = need_mesh(ctx);
  if (s != WADG_OK) return s;
  cudaSetDevice(ctx->device);
  BudgetScope budget_scope(&ctx->budget);
  if (n < 0 || (n > 0 && !xyz)) return fail(ctx, WADG_EINVAL, "bad probe list");
  ctx->probe_user.assign(xyz, xyz + 3 * (size_t)n);
  return upload_probes(ctx);
}

wadg_status wadg_set_state(wadg_ctx* ctx, const void* q, double t, int on_device) {
  wadg_status s = need_ready(ctx);
  if (s != WADG_OK) return s;
  cudaSetDevice(ctx->device);
  BudgetScope budget_scope(&ctx->budget);
  const double* qd = static_cast<const double*>(q);
  if (on_device)
    s = ctx->rs == 8 ? set_state_dev<double>(ctx, qd) : set_state_dev<float>(ctx, qd);
  else
    s = ctx->rs == 8 ? set_state_host<double>(ctx, qd) : set_state_host<float>(ctx, qd);
  if (s == WADG_OK) ctx->t = t;
  return s;
}

wadg_status wadg_get_state(wadg_ctx* ctx, void* q, double* t, int on_device) {
  wadg_status s = need_ready(ctx);
  if (s != WADG_OK) return s;
  cudaSetDevice(ctx->device);
  if (q) {
    double* qd = static_cast<double*>(q);
    if (on_device)
      s = ctx->rs == 8 ? get_state_dev<double>(ctx, qd) : get_state_dev<float>(ctx, qd);
    else
      s = ctx->rs == 8 ? get_state_host<double>(ctx, qd) : get_state_host<float>(ctx, qd);
    if (s != WADG_OK) return s;
  }
  if (t) *t = ctx->t;
  return WADG_OK;
}

wadg_status wadg_state_bytes(const wadg_ctx* ctx, size_t* bytes) {
  if (!ctx || !bytes) return fail(nullptr, WADG_EINVAL, "null argument");
  if (!ctx->has_mesh) return fail(const_cast<wadg_ctx*>(ctx), WADG_ESTATE, "no mesh set");
  size_t off[5];
  const size_t r = ctx->rs;
  *bytes = state_layout((size_t)ctx->nb * ctx->K * 6 * ctx->ref.Np * r,
                        (size_t)ctx->nb * ctx->K1 * 6 * ctx->ref.Np * r, off);
  return WADG_OK;
}

wadg_status wadg_bind_state(wadg_ctx* ctx, void* dev, size_t bytes) {
  wadg_status s = need_ready(ctx);
  if (s != WADG_OK) return s;
  if (dev && (reinterpret_cast<uintptr_t>(dev) & 255))
    return fail(ctx, WADG_EINVAL, "bound state memory must start on a 256-byte boundary");
  cudaSetDevice(ctx->device);
  BudgetScope budget_scope(&ctx->budget);
  const size_t qb = ctx->q[0].bytes, pb = ctx->p.bytes;
  size_t off[5];
  if (dev && bytes < state_layout(qb, pb, off))
    return fail(ctx, WADG_EINVAL, "the state needs %zu bytes (wadg_state_bytes), got %zu",
                state_layout(qb, pb, off), bytes);
  // the current state moves into the new buffers: copy it device to device
  DevPtr old[5];
  for (int i = 0; i < 5; ++i) {
    old[i] = *state_buf(ctx, i);
    *state_buf(ctx, i) = DevPtr{};
  }
  void* prev = ctx->bound;
  size_t prev_bytes = ctx->bound_bytes;
  ctx->bound = dev;
  ctx->bound_bytes = dev ? bytes : 0;
  s = alloc_state_buffers(ctx, qb, pb);
  if (s == WADG_OK) {
    for (int i = 0; i < 5 && s == WADG_OK; ++i) {
      DevPtr* d = state_buf(ctx, i);
      if (old[i].bytes) {
        const cudaError_t e = cudaMemcpyAsync(d->p, old[i].p, old[i].bytes,
                                              cudaMemcpyDeviceToDevice, ctx->stream);
        if (e != cudaSuccess) s = fail(ctx, WADG_ECUDA, "state copy: %s", cudaGetErrorString(e));
      }
    }
    const cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (s == WADG_OK && e != cudaSuccess)
      s = fail(ctx, WADG_ECUDA, "state copy: %s", cudaGetErrorString(e));
  }
  if (s != WADG_OK) {   // keep the old buffers
    for (int i = 0; i < 5; ++i) {
      dfree(*state_buf(ctx, i));
      *state_buf(ctx, i) = old[i];
    }
    ctx->bound = prev;
    ctx->bound_bytes = prev_bytes;
    return s;
  }
  for (int i = 0; i < 5; ++i) dfree(old[i]);
  invalidate_graphs(ctx);   // the graphs captured the old buffer addresses
  return WADG_OK;
}

wadg_status wadg_transfer_bytes(const wadg_ctx* ctx, size_t* h2d, size_t* d2h) {
  if (!ctx) return fail(nullptr, WADG_EINVAL, "null context");
  if (h2d) *h2d = ctx->h2d;
  if (d2h) *d2h = ctx->d2h;
  return WADG_OK;
}

wadg_status wadg_rk_stage(wadg_ctx* ctx, int stage, double t, double dt) {
  wadg_status s = need_mesh(ctx);
  if (s != WADG_OK) return s;
  if (stage < 0 || stage > 4) return fail(ctx, WADG_EINVAL, "stage must be 0..4");
  if ((s = need_ready(ctx)) != WADG_OK) return s;
  cudaSetDevice(ctx->device);
  s = ctx->rs == 8 ? issue_stage<double>(ctx, stage, dt, t, false)
                   : issue_stage<float>(ctx, stage, dt, t, false);
  if (s != WADG_OK) return s;
  return check_err_flag(ctx);
}

wadg_status wadg_run_steps(wadg_ctx* ctx, int64_t nsteps, double dt, double* probe_out) {
  wadg_status s = need_ready(ctx);
  if (s != WADG_OK) return s;
  if (nsteps < 0 || !(dt > 0)) return fail(ctx, WADG_EINVAL, "bad nsteps or dt");
  if (nsteps == 0) return WADG_OK;
  cudaSetDevice(ctx->device);
  BudgetScope budget_scope(&ctx->budget);
  const int64_t chunk = std::min<int64_t>(nsteps, 4096);
  const size_t need = (size_t)chunk * ctx->nprobe * 6 * ctx->nb * 8;
  if (ctx->nprobe > 0 && ctx->pr_out.bytes < need) {
    invalidate_graphs(ctx);
    CK(dalloc(ctx->pr_out, need));
  }
  if (!ctx->graph_valid || ctx->graph_dt != dt) {
    s = capture_graphs(ctx, dt);
    if (s != WADG_OK) return s;
  }
  const size_t rec = (size_t)ctx->nprobe * 6 * ctx->nb;
  int64_t done = 0;
  while (done < nsteps) {
    const int64_t n = std::min(chunk, nsteps - done);
    double tt = ctx->t + done * dt;
    CK(cudaMemcpyAsync(ctx->tdev.p, &tt, 8, cudaMemcpyHostToDevice, ctx->stream));
    ctx->h2d += 8;
    CK(cudaMemsetAsync(ctx->stepdev.p, 0, 8, ctx->stream));
    for (int64_t i = 0; i < n; ++i) {
      CK(cudaGraphLaunch(ctx->graph[ctx->cur], ctx->stream));
      ctx->cur ^= 1;
    }
    if (probe_out && rec) {
      CK(cudaMemcpyAsync(probe_out + (size_t)done * rec, ctx->pr_out.p, (size_t)n * rec * 8,
                         cudaMemcpyDeviceToHost, ctx->stream));
      ctx->d2h += (size_t)n * rec * 8;
    }
    CK(cudaStreamSynchronize(ctx->stream));
    done += n;
  }
  ctx->t += nsteps * dt;
  // a wait that gave up explains whatever the state holds: report it first
  s = check_err_flag(ctx);
  if (s != WADG_OK) return s;
  // non-finite check of the E,H state
  CK(cudaMemsetAsync(ctx->flag.p, 0, 4, ctx->stream));
  const int64_t nq = ctx->nb * ctx->K * 6 * ctx->ref.Np;
  if (ctx->rs == 8) CK(launch_check_finite<double>((const double*)ctx->q[ctx->cur].p, nq, (int*)ctx->flag.p, ctx->stream));
  else CK(launch_check_finite<float>((const float*)ctx->q[ctx->cur].p, nq, (int*)ctx->flag.p, ctx->stream));
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, ctx->flag.p, 4, cudaMemcpyDeviceToHost, ctx->stream));
  ctx->d2h += 4;
  CK(cudaStreamSynchronize(ctx->stream));
  if (flag) return fail(ctx, WADG_ENONFINITE, "state became non-finite");
  return WADG_OK;
}

wadg_status wadg_profile_stage(wadg_ctx* ctx, int reps, double dt, double* ms_out) {
  wadg_status s = need_ready(ctx);
  if (s != WADG_OK) return s;
  if (reps < 1 || !ms_out) return fail(ctx, WADG_EINVAL, "bad arguments");
  cudaSetDevice(ctx->device);
  cudaEvent_t ev[4];
  for (auto& e : ev) CK(cudaEventCreate(&e));
  float tot[2] = {0.f, 0.f};
  for (int r = 0; r < reps; ++r) {
    const int stage = r % 5;
    for (int cls = 0; cls < 2; ++cls) {
      if (cls == 1 && ctx->K1 == 0) continue;
      CK(cudaEventRecord(ev[2 * cls], ctx->stream));
      if (ctx->rs == 8) {
        StageParams<double> P = stage_params<double>(ctx, stage, dt, ctx->t, false, cls == 1);
        if (cls == 1) CK(launch_pml_class<double>(ctx, P));
        else CK(launch_stage<double>(ctx->N, false, false, P, ctx->nb, ctx->stream));
      } else {
        StageParams<float> P = stage_params<float>(ctx, stage, dt, ctx->t, false, cls == 1);
        if (cls == 1) CK(launch_pml_class<float>(ctx, P));
        else if (ctx->tc) CK(launch_stage_tc(ctx->N, false, P, ctx->nb, ctx->stream, ctx->bf16, ctx->qc));
        else CK(launch_stage<float>(ctx->N, false, false, P, ctx->nb, ctx->stream));
      }
      CK(cudaEventRecord(ev[2 * cls + 1], ctx->stream));
    }
    ctx->cur ^= 1;
    CK(cudaEventSynchronize(ev[3]));
    CK(cudaEventSynchronize(ev[1]));
    for (int cls = 0; cls < 2; ++cls) {
      if (cls == 1 && ctx->K1 == 0) continue;
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, ev[2 * cls], ev[2 * cls + 1]));
      tot[cls] += ms;
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  ms_out[0] = tot[0] / reps;
  ms_out[1] = tot[1] / reps;
  return WADG_OK;
}

}  // extern "C"

namespace {

// the E,H and P blocks of one full state (device)
struct StateBuf {
  DevPtr q, p;
};

wadg_status alloc_state(wadg_ctx* ctx, StateBuf& b) {
  CK(dalloc(b.q, ctx->q[0].bytes));
  CK(dalloc(b.p, ctx->p.bytes));
  return WADG_OK;
}
void free_state(StateBuf& b) {
  dfree(b.q);
  dfree(b.p);
}
wadg_status save_state(wadg_ctx* ctx, StateBuf& b) {
  CK(cudaMemcpyAsync(b.q.p, ctx->q[ctx->cur].p, b.q.bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  if (b.p.bytes)
    CK(cudaMemcpyAsync(b.p.p, ctx->p.p, b.p.bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  return WADG_OK;
}
wadg_status load_state(wadg_ctx* ctx, const StateBuf& b) {
  CK(cudaMemcpyAsync(ctx->q[ctx->cur].p, b.q.p, b.q.bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  if (b.p.bytes)
    CK(cudaMemcpyAsync(ctx->p.p, b.p.p, b.p.bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  return WADG_OK;
}

template <typename Real>
wadg_status adjoint_typed(wadg_ctx* ctx, int64_t nsteps, double dt, int C, double* J_out,
                          double* dJ_deps, double* dJ_dsm, double* dJ_dps) {
  const int Np = ctx->ref.Np, Nfp = ctx->ref.Nfp;
  const int64_t K = ctx->K, K1 = ctx->K1;
  const int nb = ctx->nb;
  const double t0 = ctx->t;
  const int64_t nseg = (nsteps + C - 1) / C;
  // ck: the state every C steps.  sin: the stage inputs of one segment as it
  // is recomputed, sin[5k + i - 1] = input of stage i of step k (i = 0, k = 0
  // is the checkpoint itself), sin[5n - 1] = the state at the segment's end
  std::vector<StateBuf> ck(nseg + 1), sin(5 * (size_t)std::min<int64_t>(C, nsteps));
  DevPtr lq, rq, lp, rp, G, ge, gp;
  auto cleanup = [&]() {
    for (auto& b : ck) free_state(b);
    for (auto& b : sin) free_state(b);
    for (DevPtr* d : {&lq, &rq, &lp, &rp, &G, &ge, &gp}) dfree(*d);
  };
  auto fail_clean = [&](wadg_status st) {
    cleanup();
    return st;
  };
  wadg_status st = WADG_OK;
  for (auto& b : ck) if ((st = alloc_state(ctx, b)) != WADG_OK) return fail_clean(st);
  for (auto& b : sin) if ((st = alloc_state(ctx, b)) != WADG_OK) return fail_clean(st);
  const size_t qb = ctx->q[0].bytes, pb = ctx->p.bytes;
  cudaError_t ce = cudaSuccess;
  if (ce == cudaSuccess) ce = dalloc(lq, qb);
  if (ce == cudaSuccess) ce = dalloc(rq, qb);
  if (ce == cudaSuccess) ce = dalloc(lp, pb);
  if (ce == cudaSuccess) ce = dalloc(rp, pb);
  if (ce == cudaSuccess) ce = dalloc(G, (size_t)nb * K * 4 * Nfp * 6 * sizeof(Real));
  if (ce == cudaSuccess) ce = dalloc(ge, (size_t)nb * K * 8);
  if (ce == cudaSuccess) ce = dalloc(gp, (size_t)nb * 6 * 8);
  if (ce != cudaSuccess)
    return fail_clean(fail(ctx, WADG_ENOMEM, "adjoint buffers: %s", cudaGetErrorString(ce)));

  // ---- forward pass with checkpoints every C steps; J accumulates on device
  CK(cudaMemsetAsync(ctx->obj.p, 0, ctx->obj.bytes, ctx->stream));
  if ((st = save_state(ctx, ck[0])) != WADG_OK) return fail_clean(st);
  for (int64_t sg = 0; sg < nseg; ++sg) {
    const int64_t n = std::min<int64_t>(C, nsteps - sg * C);
    double tt = t0 + sg * C * dt;
    CK(cudaMemcpyAsync(ctx->tdev.p, &tt, 8, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemsetAsync(ctx->stepdev.p, 0, 8, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int64_t i = 0; i < n; ++i) {
      CK(cudaGraphLaunch(ctx->graph[ctx->cur], ctx->stream));
      ctx->cur ^= 1;
    }
    if ((st = save_state(ctx, ck[sg + 1])) != WADG_OK) return fail_clean(st);
  }
  CK(cudaStreamSynchronize(ctx->stream));
  std::vector<double> J(nb);
  CK(cudaMemcpy(J.data(), ctx->obj.p, 8 * nb, cudaMemcpyDeviceToHost));

  // ---- reverse pass
  CK(cudaMemsetAsync(lq.p, 0, qb, ctx->stream));
  CK(cudaMemsetAsync(rq.p, 0, qb, ctx->stream));
  if (pb) {
    CK(cudaMemsetAsync(lp.p, 0, pb, ctx->stream));
    CK(cudaMemsetAsync(rp.p, 0, pb, ctx->stream));
  }
  CK(cudaMemsetAsync(ge.p, 0, ge.bytes, ctx->stream));
  CK(cudaMemsetAsync(gp.p, 0, gp.bytes, ctx->stream));
  AdjParams<Real> A{};
  A.lam_q = (Real*)lq.p; A.rho_q = (Real*)rq.p; A.lam_p = (Real*)lp.p; A.rho_p = (Real*)rp.p;
  A.G = (Real*)G.p; A.grad_eps = (double*)ge.p; A.grad_prof = (double*)gp.p;
  A.geo = (const double*)ctx->geo.p; A.fnrm = (const Real*)ctx->fnrm.p;
  A.mat = (const Real*)ctx->mat.p;
  A.nbr = (const int*)ctx->nbr.p; A.code = (const unsigned char*)ctx->code.p;
  A.sig = (const Real*)ctx->sig.p; A.ops = (const Real*)ctx->ops.p;
  {
    const int NpP = (Np + 3) & ~3, NqP = (ctx->ref.Nq + 3) & ~3;
    A.adj_ops = A.ops + 3 * Np * NpP + 4 * Nfp * NpP + Np * NqP + ctx->ref.Nq * NpP;
  }
  A.tabs = (const unsigned char*)ctx->tabs.p;
  A.strideQ = K * 6 * Np; A.strideP = K1 * 6 * Np;
  A.K = (int)K; A.K0 = (int)ctx->K0;
  A.nsrc = ctx->nsrc; A.src = (const SrcDev*)ctx->src.p; A.src_w = (const Real*)ctx->srcw.p;
  A.dt = dt; A.eps0 = ctx->has_prof ? ctx->prof.eps0 : 1.0; A.alpha = 1.0;
  A.dt_r = (Real)A.dt; A.alpha_r = (Real)A.alpha; A.inv_eps0_r = (Real)(1.0 / A.eps0);
  for (int u = 0; u < 3; ++u) {
    A.sigma_max[u] = ctx->has_prof ? ctx->prof.sigma_max[u] : 0.0;
    A.p_sigma[u] = ctx->has_prof ? ctx->prof.p_sigma[u] : 0.0;
    A.inv_sigma_max[u] = A.sigma_max[u] > 0 ? (Real)(1.0 / A.sigma_max[u]) : Real(0);
    A.inv_p_sigma[u] =
        A.sigma_max[u] > 0 && A.p_sigma[u] > 0 ? (Real)(1.0 / A.p_sigma[u]) : Real(0);
  }
  for (int64_t sg = nseg - 1; sg >= 0; --sg) {
    const int64_t s0 = sg * C, n = std::min<int64_t>(C, nsteps - s0);
    // stage input j = 5k + i of the segment (j = 5n: its end state)
    auto stage_in = [&](int64_t j) -> StateBuf& { return j == 0 ? ck[sg] : sin[j - 1]; };
    // recompute the segment from its checkpoint, each stage reading its input
    // and writing the next one in place (no copies; the Runge-Kutta register
    // restarts at every step since A_0 = 0)
    for (int64_t k = 0; k < n; ++k)
      for (int i = 0; i < 5; ++i) {
        const StateBuf& a = stage_in(5 * k + i);
        const StateBuf& b = stage_in(5 * k + i + 1);
        for (int cls = 0; cls < 2; ++cls) {
          if (cls == 1 && K1 == 0) continue;
          StageParams<Real> P = stage_params<Real>(ctx, i, dt, t0 + (s0 + k) * dt, false, cls == 1);
          P.qin = (const Real*)a.q.p;
          P.qout = (Real*)b.q.p;
          P.p = (Real*)a.p.p;
          P.pout = (Real*)b.p.p;
          if (cls == 0) CK(launch_stage<Real>(ctx->N, false, false, P, ctx->nb, ctx->stream));
          else CK(launch_pml_class<Real>(ctx, P));
        }
      }
    for (int64_t k = n - 1; k >= 0; --k) {
      const double tn = t0 + (s0 + k) * dt;
      // objective after step s0 + k: dJ/dE at the probes
      if (ctx->nprobe > 0)
        CK(launch_adjoint_probes<Real>((const Real*)stage_in(5 * k + 5).q.p, K * 6 * Np,
                                       ctx->nprobe, nb, Np, (const int*)ctx->pr_elem.p,
                                       (const double*)ctx->pr_ell.p, (Real*)lq.p, ctx->stream));
      for (int i = 4; i >= 0; --i) {
        A.q_in = (const Real*)stage_in(5 * k + i).q.p;
        A.p_in = (const Real*)stage_in(5 * k + i).p.p;
        A.rk_a = kRkA[i];
        A.rk_b = kRkB[i];
        A.rk_a_r = (Real)A.rk_a;
        A.rk_b_r = (Real)A.rk_b;
        A.t = tn + kRkC.c[i] * dt;
        CK(launch_adjoint_stage<Real>(ctx->N, A, nb, ctx->stream, ctx->qc));
      }
    }
  }
  CK(cudaStreamSynchronize(ctx->stream));
  // final forward state back in place
  if ((st = load_state(ctx, ck[nseg])) != WADG_OK) return fail_clean(st);
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->t = t0 + nsteps * dt;
  std::vector<double> hge((size_t)nb * K), hgp((size_t)nb * 6);
  CK(cudaMemcpy(hge.data(), ge.p, ge.bytes, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(hgp.data(), gp.p, gp.bytes, cudaMemcpyDeviceToHost));
  cleanup();
  // d/d eps_r: eps_r enters through eps = eps_r (normalised units)
  if (J_out) for (int b = 0; b < nb; ++b) J_out[b] = J[b];
  if (dJ_deps)
    for (int b = 0; b < nb; ++b)
      for (int64_t e = 0; e < K; ++e) dJ_deps[(size_t)b * K + ctx->perm[e]] = hge[(size_t)b * K + e];
  for (int b = 0; b < nb; ++b)
    for (int u = 0; u < 3; ++u) {
      if (dJ_dsm) dJ_dsm[b * 3 + u] = hgp[b * 6 + u];
      if (dJ_dps) dJ_dps[b * 3 + u] = hgp[b * 6 + 3 + u];
    }
  return WADG_OK;
}

}  // namespace

extern "C" {

wadg_status wadg_adjoint(wadg_ctx* ctx, int64_t nsteps, double dt, int32_t ckpt_every,
                         double* J_out, double* dJ_deps, double* dJ_dsigma_max,
                         double* dJ_dp_sigma) {
  wadg_status s = need_ready(ctx);
  if (s != WADG_OK) return s;
  if (nsteps < 1 || !(dt > 0) || ckpt_every < 1) return fail(ctx, WADG_EINVAL, "bad arguments");
  if (ctx->tc) return fail(ctx, WADG_EUNSUPPORTED, "the adjoint runs on the FP64/FP32 kernels");
  if (ctx->kappa) return fail(ctx, WADG_EUNSUPPORTED, "the adjoint is built for kappa = 1");
  if (ctx->scheme != WADG_PML_WAA)
    return fail(ctx, WADG_EUNSUPPORTED, "the adjoint is built for the weight-adjusted scheme");
  if (ctx->nprobe < 1) return fail(ctx, WADG_ESTATE, "the objective needs probes");
  cudaSetDevice(ctx->device);
  BudgetScope budget_scope(&ctx->budget);
  const size_t need = (size_t)std::min<int64_t>(ckpt_every, 4096) * ctx->nprobe * 6 * ctx->nb * 8;
  if (ctx->pr_out.bytes < need) {
    invalidate_graphs(ctx);
    CK(dalloc(ctx->pr_out, need));
  }
  if (!ctx->graph_valid || ctx->graph_dt != dt) {
    s = capture_graphs(ctx, dt);
    if (s != WADG_OK) return s;
  }
  const int C = (int)std::min<int64_t>(ckpt_every, 4096);
  return ctx->rs == 8
             ? adjoint_typed<double>(ctx, nsteps, dt, C, J_out, dJ_deps, dJ_dsigma_max, dJ_dp_sigma)
             : adjoint_typed<float>(ctx, nsteps, dt, C, J_out, dJ_deps, dJ_dsigma_max, dJ_dp_sigma);
}

wadg_status wadg_stable_dt(const wadg_ctx* ctx, double cfl, double* dt_out) {
  if (!ctx || !dt_out) return fail(nullptr, WADG_EINVAL, "null argument");
  if (!ctx->has_mesh) return fail(const_cast<wadg_ctx*>(ctx), WADG_ESTATE, "no mesh set");
  *dt_out = cfl * 2.0 / ((ctx->N + 1.0) * (ctx->N + 1.0) * ctx->fscale_max);
  return WADG_OK;
}

wadg_status wadg_objective(wadg_ctx* ctx, double* J_out) {
  if (!ctx || !J_out) return fail(nullptr, WADG_EINVAL, "null argument");
  cudaSetDevice(ctx->device);
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaMemcpy(J_out, ctx->obj.p, 8 * (size_t)ctx->nb, cudaMemcpyDeviceToHost));
  ctx->d2h += 8 * (size_t)ctx->nb;
  return WADG_OK;
}

wadg_status wadg_memory_report(const wadg_ctx* ctx, size_t* bytes_state, size_t* bytes_pml_coeff,
                               size_t* bytes_operators, size_t* bytes_geometry) {
  if (!ctx) return fail(nullptr, WADG_EINVAL, "null context");
  if (bytes_state) *bytes_state = ctx->q[0].bytes + ctx->q[1].bytes + ctx->rq.bytes + ctx->p.bytes + ctx->rp.bytes;
  if (bytes_pml_coeff)
    *bytes_pml_coeff = ctx->scheme == WADG_PML_STORED ? ctx->stored.bytes
                                                       : ctx->sig.bytes + ctx->kap.bytes;
  if (bytes_operators) *bytes_operators = ctx->ops.bytes + ctx->tabs.bytes;
  if (bytes_geometry)
    *bytes_geometry = ctx->geo.bytes + ctx->geof.bytes + ctx->fnrm.bytes + ctx->mat.bytes +
                      ctx->nbr.bytes + ctx->code.bytes;
  return WADG_OK;
}

wadg_status wadg_mesh_info(const wadg_ctx* ctx, int64_t* K, int64_t* K_pml, int32_t* Np,
                           int32_t* Nq) {
  if (!ctx) return fail(nullptr, WADG_EINVAL, "null context");
  if (K) *K = ctx->K;
  if (K_pml) *K_pml = ctx->K1;
  if (Np) *Np = ctx->ref.Np;
  if (Nq) *Nq = ctx->ref.Nq_rule;
  return WADG_OK;
}

wadg_status wadg_synchronize(wadg_ctx* ctx) {
  if (!ctx) return fail(nullptr, WADG_EINVAL, "null context");
  cudaSetDevice(ctx->device);
  CK(cudaStreamSynchronize(ctx->stream));
  return WADG_OK;
}

wadg_status wadg_set_memory_limit(wadg_ctx* ctx, size_t bytes, size_t* held_out) {
  if (!ctx) return fail(nullptr, WADG_EINVAL, "null context");
  ctx->budget.limit = bytes;
  if (held_out) *held_out = ctx->budget.held;
  return WADG_OK;
}

wadg_status wadg_arm_wait_timeout(wadg_ctx* ctx) {
  if (!ctx) return fail(nullptr, WADG_EINVAL, "null context");
  if (!ctx->tc)
    return fail(ctx, WADG_EUNSUPPORTED, "only the tensor-core kernels wait on device-side signals");
  cudaSetDevice(ctx->device);
  const int one = 1;
  CK(cudaMemcpyAsync((int*)ctx->errflag.p + 1, &one, 4, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return WADG_OK;
}

wadg_status wadg_reference_operator(int N, int which, double* out, int64_t cap, int64_t* n_out) {
  RefOps R;
  const char* e = nullptr;
  if (!build_ref_ops(N, R, &e)) return fail(nullptr, WADG_EINVAL, "%s", e);
  std::vector<double> v;
  switch (which) {
    case 0: v = R.Dr; break;
    case 1: v = R.Ds; break;
    case 2: v = R.Dt; break;
    case 3: v = R.LIFT; break;
    case 4: v = R.Vq; break;
    case 5: v = R.Pq; break;
    case 6:
      for (int q = 0; q < R.Nq; ++q) v.insert(v.end(), {R.rq[q], R.sq[q], R.tq[q], R.wq[q]});
      break;
    case 7: v = R.Minv; break;
    default: return fail(nullptr, WADG_EINVAL, "unknown operator %d", which);
  }
  if (n_out) *n_out = (int64_t)v.size();
  if (!out) return WADG_OK;
  if (cap < (int64_t)v.size()) return fail(nullptr, WADG_EINVAL, "capacity %lld < %zu", (long long)cap, v.size());
  std::memcpy(out, v.data(), v.size() * 8);
  return WADG_OK;
}

const char* wadg_last_error(const wadg_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_err.c_str();
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Stepping without device allocation (wadg_run_steps_noalloc).
//
// wadg_run_steps may allocate on first use (the device staging area of the
// probe records, the CUDA graphs of a step).  Callers that must not allocate
// device memory at that point use wadg_run_steps_noalloc instead: it launches
// the stage kernels one by one and keeps its scratch -- the device time and
// step counters the kernels read, the non-finite flag and the probe records
// of a chunk of steps before they are copied to the host -- in the file-scope
// array below.  The array is part of the library image: every GPU that loads
// the library holds its kNoAllocBytes until the process exits.  In host code
// the array's name is only a stand-in for the device object; each call looks
// up its device address on the current device with cudaGetSymbolAddress.
// With lazy module loading the array's memory is committed when the module is
// first used on a device, so the first call should come before any stream
// capture.
namespace {

constexpr size_t kNoAllocBytes = size_t(16) << 20;   // 16 MiB per device
constexpr size_t kNoAllocRecords = 256;               // offset of the probe records
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// device address of the scratch array on ctx's device (which is current).
// Looked up on every call rather than cached: the lookup is cheap once the
// module is loaded, and an address kept from before a device reset or a
// recreated primary context would be stale.
wadg_status noalloc_scratch(wadg_ctx* ctx, unsigned char** out) {
  void* a = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&a, g_noalloc_scratch);
  if (e != cudaSuccess || !a)
    return fail(ctx, WADG_ECUDA, "cudaGetSymbolAddress of the step scratch: %s",
                cudaGetErrorString(e));
  *out = static_cast<unsigned char*>(a);
  return WADG_OK;
}

template <typename Real>
wadg_status noalloc_stage(wadg_ctx* ctx, int stage, double dt, const double* tdev) {
  if (ctx->tc) {
    StageParams<float> A = stage_params<float>(ctx, stage, dt, 0.0, false, false);
    A.t_dev = tdev;
    CK(launch_stage_tc(ctx->N, false, A, ctx->nb, ctx->stream, ctx->bf16, ctx->qc));
    if (ctx->K1 > 0) {
      StageParams<float> B = stage_params<float>(ctx, stage, dt, 0.0, false, true);
      B.t_dev = tdev;
      CK(launch_pml_class<float>(ctx, B));
    }
  } else {
    StageParams<Real> A = stage_params<Real>(ctx, stage, dt, 0.0, false, false);
    A.t_dev = tdev;
    CK(launch_stage<Real>(ctx->N, false, false, A, ctx->nb, ctx->stream));
    if (ctx->K1 > 0) {
      StageParams<Real> B = stage_params<Real>(ctx, stage, dt, 0.0, false, true);
      B.t_dev = tdev;
      CK(launch_pml_class<Real>(ctx, B));
    }
  }
  ctx->cur ^= 1;
  return WADG_OK;
}

}  // namespace

extern "C" wadg_status wadg_run_steps_noalloc(wadg_ctx* ctx, int64_t nsteps, double dt,
                                              double* probe_out) {
  wadg_status s = need_ready(ctx);
  if (s != WADG_OK) return s;
  if (nsteps < 0 || !(dt > 0)) return fail(ctx, WADG_EINVAL, "bad nsteps or dt");
  if (nsteps == 0) return WADG_OK;
  cudaSetDevice(ctx->device);
  unsigned char* scr = nullptr;
  if ((s = noalloc_scratch(ctx, &scr)) != WADG_OK) return s;
  double* tdev = reinterpret_cast<double*>(scr);
  int64_t* stepdev = reinterpret_cast<int64_t*>(scr + 8);
  int* flag = reinterpret_cast<int*>(scr + 16);
  double* rec_dev = reinterpret_cast<double*>(scr + kNoAllocRecords);
  const size_t rec = (size_t)ctx->nprobe * 6 * ctx->nb;   // doubles per step
  const size_t cap = (kNoAllocBytes - kNoAllocRecords) / 8;
  if (rec > cap)
    return fail(ctx, WADG_EINVAL,
                "probe records of one step (%zu bytes) exceed the %zu-byte step scratch",
                rec * 8, cap * 8);
  const int64_t chunk = rec ? std::min<int64_t>(nsteps, (int64_t)(cap / rec)) : nsteps;
  int64_t done = 0;
  while (done < nsteps) {
    const int64_t n = std::min(chunk, nsteps - done);
    // the array keeps the previous call's contents: set the counters
    const double tt = ctx->t + done * dt;
    CK(cudaMemcpyAsync(tdev, &tt, 8, cudaMemcpyHostToDevice, ctx->stream));
    ctx->h2d += 8;
    CK(cudaMemsetAsync(stepdev, 0, 8, ctx->stream));
    for (int64_t i = 0; i < n; ++i) {
      for (int st = 0; st < 5; ++st) {
        s = ctx->rs == 8 ? noalloc_stage<double>(ctx, st, dt, tdev)
                         : noalloc_stage<float>(ctx, st, dt, tdev);
        if (s != WADG_OK) return s;
      }
      if (ctx->nprobe > 0) {
        ProbeParams pp{};
        pp.q = ctx->q[ctx->cur].p;
        pp.strideQ = ctx->K * 6 * ctx->ref.Np;
        pp.nprobe = ctx->nprobe;
        pp.nb = ctx->nb;
        pp.Np = ctx->ref.Np;
        pp.elem = (const int*)ctx->pr_elem.p;
        pp.ell = (const double*)ctx->pr_ell.p;
        pp.out = rec_dev;
        pp.obj = (double*)ctx->obj.p;
        pp.step = stepdev;
        CK(launch_probes(ctx->rs == 8, pp, ctx->stream));
      }
      CK(launch_advance(tdev, stepdev, dt, ctx->stream));
    }
    if (probe_out && rec) {
      CK(cudaMemcpyAsync(probe_out + (size_t)done * rec, rec_dev, (size_t)n * rec * 8,
                         cudaMemcpyDeviceToHost, ctx->stream));
      ctx->d2h += (size_t)n * rec * 8;
    }
    CK(cudaStreamSynchronize(ctx->stream));
    done += n;
  }
  ctx->t += nsteps * dt;
  // a wait that gave up explains whatever the state holds: report it first
  if ((s = check_err_flag(ctx)) != WADG_OK) return s;
  CK(cudaMemsetAsync(flag, 0, 4, ctx->stream));
  const int64_t nq = ctx->nb * ctx->K * 6 * ctx->ref.Np;
  if (ctx->rs == 8) CK(launch_check_finite<double>((const double*)ctx->q[ctx->cur].p, nq, flag, ctx->stream));
  else CK(launch_check_finite<float>((const float*)ctx->q[ctx->cur].p, nq, flag, ctx->stream));
  int hflag = 0;
  CK(cudaMemcpyAsync(&hflag, flag, 4, cudaMemcpyDeviceToHost, ctx->stream));
  ctx->d2h += 4;
  CK(cudaStreamSynchronize(ctx->stream));
  if (hflag) return fail(ctx, WADG_ENONFINITE, "state became non-finite");
  return WADG_OK;
}

// ====================================================================== groups
// Several contexts (meshes of any size and order, FP32 CUDA-core kernels)
// advanced together: every Runge-Kutta stage of every member is one launch of
// group_stage_kernel; its blocks start on the (member, element class) items in
// proportion to the work and then take tiles from per-item counters until
// none are left (dynamic balancing); one step (5 launches plus each member's
// probe and clock kernels) is captured in a CUDA graph.
struct wadg_group {
  std::vector<wadg_ctx*> ctx;
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  int sms = 1;
  int blocks_per_sm = 1;   // autotuned
  int tile_div = 1;        // autotuned: tile = largest tile / tile_div
  // the grouped variant kernels serve FP32 CUDA-core members with the
  // (N+1)^3 rule and a weight-adjusted or element-constant PML; any other
  // member (FP64, TF32, BF16, a compact rule, the stored scheme) makes the
  // group launch per item
  bool variants_ok = true;
  std::vector<double> dt_now;   // the members' steps of the current tables
  bool per_item = false;   // autotuned: each (member, class) item launched as its
                           // single-context kernel (else one grouped kernel per variant)
  bool parallel = true;    // autotuned: a stage's launches on parallel branches
  bool share = false;      // autotuned: a variant's grid is its share of the GPU (by
                           // algorithmic flops) instead of the whole GPU
  int nblocks = 0;         // all variants
  struct Item { int c; bool pml; int code; int tile; int64_t tiles; double work; };
  std::vector<Item> items;   // sorted by variant code
  // a variant: the items [off, off + n) of one code, its kernel's shared
  // memory and grid, and its block split first[foff .. foff + n]
  struct Variant { int code; int off, n; size_t smem; int nblocks; int foff; };
  std::vector<Variant> vars;
  std::vector<int> first;
  DevPtr dparams, dfirst;          // params [2 parities][5 stages][items]
  DevPtr dntiles, dcounter;        // tiles per item, tile counters (zeroed per launch)
  // streams and events of the parallel branches (variant v > 0 on aux[v - 1])
  std::vector<cudaStream_t> aux;
  std::vector<cudaEvent_t> ev;     // ev[0] fork, ev[v] join of variant v
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  // what the graphs were built for: each member's generation, step size and
  // buffer parity (a later call with the same generations and steps reuses
  // them from the matching parity)
  std::vector<uint64_t> built_gen;
  std::vector<double> built_dt;
  std::vector<int> built_cur;
  // L2 clusters: the members packed so that each cluster's per-step data fits
  // half of the L2, each cluster advanced through all the steps of a call
  // before the next (members are independent, so only the order in time
  // changes: a small member's state then stays in L2 from step to step);
  // members larger than that form one cluster.  Empty when one cluster would
  // hold every member.
  std::vector<std::vector<int>> cluster_of;
  std::vector<wadg_group*> clusters;
};

namespace {

wadg_status gfail(wadg_group* g, wadg_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g->err = buf;
  return s;
}

#define GCK(call)                                                                       \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return gfail(g, e_ == cudaErrorMemoryAllocation ? WADG_ENOMEM : WADG_ECUDA,       \
                   "%s: %s", #call, cudaGetErrorString(e_));                            \
  } while (0)

// every member's device tables are complete (no set-up call of a member
// failed part-way since its last success)
wadg_status group_members_ready(wadg_group* g) {
  for (size_t c = 0; c < g->ctx.size(); ++c) {
    const wadg_ctx* x = g->ctx[c];
    if (!x->has_mesh || !x->ready || !x->src_ok || !x->probes_ok || !x->ops_ok)
      return gfail(g, WADG_ESTATE, "member %d has an incomplete set-up (a set-up call failed)",
                   (int)c);
  }
  return WADG_OK;
}

void group_drop_graphs(wadg_group* g) {
  for (auto& x : g->graph)
    if (x) { cudaGraphExecDestroy(x); x = nullptr; }
  g->built_gen.clear();
}

// per-element flops of a stage (the algorithmic count used by the benchmark),
// the weight of a work item in the block split
double item_cost(int N, bool pml) {
  const double Np = (N + 1) * (N + 2) * (N + 3) / 6.0, Nfp = (N + 1) * (N + 2) / 2.0;
  const double Nq = (N + 1.0) * (N + 1.0) * (N + 1.0);
  double f = 36 * Np * Np + 90 * Np + 240 * Nfp + 48 * Np * Nfp + 24 * Np;
  if (pml) f += 48 * Nq * Np + 24 * Nq + 36 * Np;
  return f;
}

// work items (sorted by variant), tile sizes, and each variant's grid and
// block split for the current tuning.  A variant's grid fills the GPU at its
// own occupancy: its blocks run as long as its tiles last, and the SMs they
// leave go to the other variants of the stage (parallel graph branches).
void group_plan(wadg_group* g) {
  g->items.clear();
  for (int c = 0; c < (int)g->ctx.size(); ++c) {
    wadg_ctx* x = g->ctx[c];
    for (int cls = 0; cls < 2; ++cls) {
      const int64_t ne = cls == 0 ? x->K0 : x->K1;
      if (ne == 0) continue;
      const bool pml = cls == 1;
      wadg_group::Item it;
      it.c = c;
      it.pml = pml;
      it.code = x->N * 4 + (pml ? (x->kappa ? 2 : 1) : 0);
      const int tmax = g->variants_ok ? group_tile_max(x->N, pml) : 1;
      it.tile = std::max(1, tmax / g->tile_div);
      it.tiles = (ne + it.tile - 1) / it.tile * x->nb;
      it.work = item_cost(x->N, pml) * (double)ne * x->nb;
      g->items.push_back(it);
    }
  }
  // heaviest variants first: their launches are issued first
  std::map<int, double> vwork;
  for (auto& it : g->items) vwork[it.code] += it.work;
  std::stable_sort(g->items.begin(), g->items.end(), [&](const auto& a, const auto& b) {
    return a.code != b.code && (vwork[a.code] > vwork[b.code] ||
                                (vwork[a.code] == vwork[b.code] && a.code < b.code));
  });
  g->vars.clear();
  g->first.clear();
  g->nblocks = 0;
  if (!g->variants_ok) {   // per-item launches only; tiles as each kernel chooses
    g->per_item = true;
    for (auto& it : g->items) it.tile = 0;
    return;
  }
  double all = 0.0;
  for (auto& it : g->items) all += it.work;
  all = std::max(all, 1.0);
  for (int i = 0; i < (int)g->items.size();) {
    wadg_group::Variant v{};
    v.code = g->items[i].code;
    v.off = i;
    while (i < (int)g->items.size() && g->items[i].code == v.code) ++i;
    v.n = i - v.off;
    double tot = 0.0;
    for (int j = v.off; j < i; ++j) {
      const auto& it = g->items[j];
      v.smem = std::max(v.smem, group_smem_bytes(it.code / 4, it.pml, it.tile));
      tot += it.work;
    }
    const int bps = std::max(1, std::min(g->blocks_per_sm, group_blocks_per_sm(v.code, v.smem)));
    const int want = g->share ? std::max(1, (int)std::lround(bps * g->sms * tot / all))
                              : bps * g->sms;
    v.foff = (int)g->first.size();
    g->first.push_back(0);
    for (int j = v.off; j < i; ++j) {
      const auto& it = g->items[j];
      int64_t nb = (int64_t)std::llround(want * it.work / std::max(tot, 1.0));
      nb = std::max<int64_t>(1, std::min<int64_t>(nb, it.tiles));
      g->first.push_back(g->first.back() + (int)nb);
    }
    v.nblocks = g->first.back();
    g->nblocks += v.nblocks;
    g->vars.push_back(v);
  }
}

// the streams and events of the parallel branches
wadg_status group_branches(wadg_group* g) {
  const size_t want = std::max(g->vars.size(), std::min<size_t>(g->items.size(), 8));
  while (g->aux.size() + 1 < want) {
    cudaStream_t st;
    GCK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    g->aux.push_back(st);
  }
  while (g->ev.size() < std::max<size_t>(1, want)) {
    cudaEvent_t e;
    GCK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    g->ev.push_back(e);
  }
  return WADG_OK;
}

// device bytes a member reads or writes in a step
size_t member_step_bytes(const wadg_ctx* x) {
  return 2 * x->q[0].bytes + x->rq.bytes + x->p.bytes + x->rp.bytes + x->sig.bytes + x->kap.bytes +
         x->geo.bytes + x->fnrm.bytes + x->mat.bytes + x->nbr.bytes + x->code.bytes;
}

// members packed into clusters of at most half the L2 (smallest first);
// members above that go together into a last cluster
std::vector<std::vector<int>> group_clusters(const wadg_group* g) {
  int l2 = 0;
  cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, g->device);
  const size_t budget = (size_t)std::max(l2, 0) / 2;
  std::vector<int> order(g->ctx.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return member_step_bytes(g->ctx[a]) < member_step_bytes(g->ctx[b]);
  });
  std::vector<std::vector<int>> cl;
  std::vector<int> open, large;
  size_t used = 0;
  for (int m : order) {
    const size_t b = member_step_bytes(g->ctx[m]);
    if (b > budget) {
      large.push_back(m);
      continue;
    }
    if (used + b > budget && !open.empty()) {
      cl.push_back(open);
      open.clear();
      used = 0;
    }
    open.push_back(m);
    used += b;
  }
  if (!open.empty()) cl.push_back(open);
  if (!large.empty()) cl.push_back(large);
  if (cl.size() <= 1) cl.clear();
  for (auto& c : cl) std::sort(c.begin(), c.end());
  return cl;
}

void group_drop_clusters(wadg_group* g);

// stage parameters of every item for both step parities and all 5 stages
wadg_status group_upload(wadg_group* g, const double* dt) {
  g->dt_now.assign(dt, dt + g->ctx.size());
  if (!g->variants_ok) return group_branches(g);
  const int ni = (int)g->items.size();
  std::vector<StageParams<float>> hp((size_t)2 * 5 * ni);
  std::vector<int> cur0(g->ctx.size());
  for (size_t c = 0; c < g->ctx.size(); ++c) cur0[c] = g->ctx[c]->cur;
  for (int par = 0; par < 2; ++par)
    for (int st = 0; st < 5; ++st)
      for (int i = 0; i < ni; ++i) {
        const auto& it = g->items[i];
        wadg_ctx* x = g->ctx[it.c];
        // every stage flips a member's buffers; a step (5 stages) flips them once
        x->cur = cur0[it.c] ^ par ^ (st & 1);
        StageParams<float> P = stage_params<float>(x, st, dt[it.c], 0.0, true, it.pml);
        P.nb = x->nb;
        P.tile_elems = it.tile;
        hp[((size_t)par * 5 + st) * ni + i] = P;
        x->cur = cur0[it.c];
      }
  std::vector<int> ntiles(ni);
  for (int i = 0; i < ni; ++i) ntiles[i] = (int)g->items[i].tiles;
  GCK(dalloc(g->dntiles, ntiles.size() * sizeof(int)));
  GCK(dalloc(g->dcounter, ntiles.size() * sizeof(int)));
  GCK(cudaMemcpy(g->dntiles.p, ntiles.data(), ntiles.size() * sizeof(int), cudaMemcpyHostToDevice));
  GCK(dalloc(g->dparams, hp.size() * sizeof(StageParams<float>)));
  GCK(dalloc(g->dfirst, g->first.size() * sizeof(int)));
  GCK(cudaMemcpy(g->dparams.p, hp.data(), hp.size() * sizeof(StageParams<float>),
                 cudaMemcpyHostToDevice));
  GCK(cudaMemcpy(g->dfirst.p, g->first.data(), g->first.size() * sizeof(int),
                 cudaMemcpyHostToDevice));
  return group_branches(g);
}

GroupParams group_params(wadg_group* g, const wadg_group::Variant& v, int par, int st) {
  GroupParams G{};
  G.p = (const StageParams<float>*)g->dparams.p + ((size_t)par * 5 + st) * g->items.size() + v.off;
  G.first = (const int*)g->dfirst.p + v.foff;
  G.ntiles = (const int*)g->dntiles.p + v.off;
  G.counter = (int*)g->dcounter.p + v.off;
  G.nitems = v.n;
  return G;
}

// one stage with per-item launches: every (member, class) item as its
// single-context kernel with its own parameters, spread over up to 8
// parallel branches (or all on the group's stream)
cudaError_t group_launch_items(wadg_group* g, int par, int st) {
  const size_t ni = g->items.size();
  const size_t nbr = g->parallel ? std::min<size_t>(ni, g->aux.size() + 1) : 1;
  cudaError_t e = cudaSuccess;
  if (nbr > 1) {
    if ((e = cudaEventRecord(g->ev[0], g->stream)) != cudaSuccess) return e;
    for (size_t k = 1; k < nbr; ++k)
      if ((e = cudaStreamWaitEvent(g->aux[k - 1], g->ev[0], 0)) != cudaSuccess) return e;
  }
  for (size_t i = 0; i < ni; ++i) {
    const auto& it = g->items[i];
    wadg_ctx* x = g->ctx[it.c];
    const size_t k = i % nbr;
    cudaStream_t s = k == 0 ? g->stream : g->aux[k - 1];
    // the buffers of this parity and stage (each stage flips them, a step once)
    const int cur0 = x->cur;
    x->cur = cur0 ^ par ^ (st & 1);
    e = launch_member_class(x, st, g->dt_now[it.c], it.pml, it.tile, s);
    x->cur = cur0;
    if (e != cudaSuccess) return e;
  }
  for (size_t k = 1; k < nbr; ++k) {
    if ((e = cudaEventRecord(g->ev[k], g->aux[k - 1])) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(g->stream, g->ev[k], 0)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// one grouped stage: clear the tile counters, then one launch per variant,
// variant 0 on the group's stream and the others on parallel branches that
// fork from it after the clear and join it before the next stage
cudaError_t group_launch(wadg_group* g, int par, int st) {
  if (g->per_item) return group_launch_items(g, par, st);
  cudaError_t e = cudaMemsetAsync(g->dcounter.p, 0, g->items.size() * sizeof(int), g->stream);
  if (e != cudaSuccess) return e;
  const size_t nv = g->vars.size();
  const bool fork = g->parallel && nv > 1;
  if (fork) {
    if ((e = cudaEventRecord(g->ev[0], g->stream)) != cudaSuccess) return e;
    for (size_t v = 1; v < nv; ++v)
      if ((e = cudaStreamWaitEvent(g->aux[v - 1], g->ev[0], 0)) != cudaSuccess) return e;
  }
  for (size_t v = 0; v < nv; ++v) {
    const auto& V = g->vars[v];
    cudaStream_t s = v == 0 || !fork ? g->stream : g->aux[v - 1];
    e = launch_group_stage(V.code, group_params(g, V, par, st), V.nblocks, V.smem, s);
    if (e != cudaSuccess) return e;
  }
  for (size_t v = 1; fork && v < nv; ++v) {
    if ((e = cudaEventRecord(g->ev[v], g->aux[v - 1])) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(g->stream, g->ev[v], 0)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// one step of parity par: 5 grouped stage launches, then every member's probes
// and clock
wadg_status group_issue_step(wadg_group* g, int par, const double* dt) {
  for (int st = 0; st < 5; ++st) GCK(group_launch(g, par, st));
  for (size_t c = 0; c < g->ctx.size(); ++c) {
    wadg_ctx* x = g->ctx[c];
    if (x->nprobe > 0) {
      ProbeParams pp{};
      pp.q = x->q[x->cur ^ par ^ 1].p;   // the step's output buffer
      pp.strideQ = x->K * 6 * x->ref.Np;
      pp.nprobe = x->nprobe;
      pp.nb = x->nb;
      pp.Np = x->ref.Np;
      pp.elem = (const int*)x->pr_elem.p;
      pp.ell = (const double*)x->pr_ell.p;
      pp.out = (double*)x->pr_out.p;
      pp.obj = (double*)x->obj.p;
      pp.step = (const int64_t*)x->stepdev.p;
      GCK(launch_probes(x->rs == 8, pp, g->stream));
    }
    GCK(launch_advance((double*)x->tdev.p, (int64_t*)x->stepdev.p, dt[c], g->stream));
  }
  return WADG_OK;
}

wadg_status group_capture(wadg_group* g, const double* dt) {
  group_drop_graphs(g);
  for (int par = 0; par < 2; ++par) {
    cudaGraph_t graph;
    GCK(cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal));
    wadg_status st = group_issue_step(g, par, dt);
    cudaError_t e = cudaStreamEndCapture(g->stream, &graph);
    if (st != WADG_OK) return st;
    GCK(e);
    e = cudaGraphInstantiate(&g->graph[par], graph, 0);
    cudaGraphDestroy(graph);
    GCK(e);
  }
  return WADG_OK;
}

}  // namespace

extern "C" {

wadg_status wadg_group_create(int32_t n, wadg_ctx* const* ctxs, wadg_group** out) {
  if (!out || n < 1 || !ctxs) return fail(nullptr, WADG_EINVAL, "bad group arguments");
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    wadg_ctx* x = ctxs[i];
    if (!x) return fail(nullptr, WADG_EINVAL, "null context %d", i);
    if (!x->has_mesh || !x->ready || !x->src_ok || !x->probes_ok || !x->ops_ok)
      return fail(nullptr, WADG_ESTATE, "context %d has no mesh or an incomplete set-up", i);
    if (x->device != ctxs[0]->device)
      return fail(nullptr, WADG_EINVAL, "group members must share a device");
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == x) return fail(nullptr, WADG_EINVAL, "context %d listed twice", i);
  }
  wadg_group* g = new wadg_group();
  g->ctx.assign(ctxs, ctxs + n);
  for (int i = 0; i < n; ++i) {
    const wadg_ctx* x = ctxs[i];
    if (x->prec != WADG_FP32 || x->tc || x->qc != 0 || x->scheme == WADG_PML_STORED)
      g->variants_ok = false;
  }
  g->device = ctxs[0]->device;
  g->stream = ctxs[0]->stream;
  cudaSetDevice(g->device);
  cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, g->device);
  if (g->sms < 1) g->sms = 1;
  cudaError_t e = configure_group_kernel();
  if (e != cudaSuccess) {
    delete g;
    return fail(nullptr, WADG_ECUDA, "group kernel set-up: %s", cudaGetErrorString(e));
  }
  g->blocks_per_sm = 2;   // capped per variant by its occupancy
  group_plan(g);
  *out = g;
  return WADG_OK;
}

wadg_status wadg_group_destroy(wadg_group* g) {
  if (!g) return WADG_OK;
  cudaSetDevice(g->device);
  group_drop_clusters(g);
  group_drop_graphs(g);
  dfree(g->dparams);
  dfree(g->dfirst);
  dfree(g->dntiles);
  dfree(g->dcounter);
  for (cudaStream_t st : g->aux) cudaStreamDestroy(st);
  for (cudaEvent_t e : g->ev) cudaEventDestroy(e);
  delete g;
  return WADG_OK;
}

wadg_status wadg_group_autotune(wadg_group* g, const double* dt, int32_t reps, double* ms_out) {
  if (!g) return WADG_EINVAL;
  if (!dt || reps < 1) return gfail(g, WADG_EINVAL, "bad arguments");
  if (wadg_status s0 = group_members_ready(g); s0 != WADG_OK) return s0;
  cudaSetDevice(g->device);
  group_drop_graphs(g);
  cudaEvent_t e0, e1;
  GCK(cudaEventCreate(&e0));
  GCK(cudaEventCreate(&e1));
  double best = 1e300;
  int best_bps = 1, best_div = 1;
  bool best_par = true, best_share = false, best_item = false;
  for (int item = g->variants_ok ? 0 : 1; item < 2; ++item)
  for (int par = 1; par >= 0; --par)
  for (int shr = 0; shr < (item ? 1 : 2); ++shr)
  for (int div : {1, 2, 4}) {
    if (!g->variants_ok && div > 1) continue;   // per-item launches keep each kernel's tile
    g->per_item = item != 0;
    g->parallel = par != 0;
    g->share = shr != 0;
    g->tile_div = div;
    g->blocks_per_sm = 1;
    group_plan(g);
    int occ = 1;   // the most blocks per SM any variant can hold (per-item: the
                   // single-context launcher sizes its own grid)
    if (!item)
      for (const auto& v : g->vars) occ = std::max(occ, group_blocks_per_sm(v.code, v.smem));
    for (int bps = 1; bps <= std::min(occ, 4); ++bps) {
      g->blocks_per_sm = bps;
      group_plan(g);
      wadg_status s = group_upload(g, dt);
      if (s != WADG_OK) return s;
      for (int st = 0; st < 5; ++st) GCK(group_launch(g, 0, st));   // one untimed step
      GCK(cudaEventRecord(e0, g->stream));
      for (int r = 0; r < reps; ++r) GCK(group_launch(g, 0, r % 5));
      GCK(cudaEventRecord(e1, g->stream));
      GCK(cudaEventSynchronize(e1));
      float ms = 0.f;
      GCK(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) {
        best = ms; best_bps = bps; best_div = div; best_par = g->parallel; best_share = g->share;
        best_item = g->per_item;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  g->blocks_per_sm = best_bps;
  g->tile_div = best_div;
  g->parallel = best_par;
  g->share = best_share;
  g->per_item = best_item;
  group_plan(g);
  if (ms_out) *ms_out = best / reps;
  return WADG_OK;
}

wadg_status wadg_group_set_tuning(wadg_group* g, int32_t per_item, int32_t parallel,
                                  int32_t share, int32_t tile_divisor, int32_t blocks_per_sm) {
  if (!g) return WADG_EINVAL;
  if (tile_divisor < 1 || tile_divisor > 64 || blocks_per_sm < 1 || blocks_per_sm > 8)
    return gfail(g, WADG_EINVAL, "tile divisor must be 1..64 and blocks per SM 1..8");
  if (!per_item && !g->variants_ok)
    return gfail(g, WADG_EUNSUPPORTED,
                 "the grouped variant kernels serve FP32 CUDA-core members with the (N+1)^3 "
                 "rule and a weight-adjusted or element-constant PML only");
  group_drop_graphs(g);
  g->per_item = per_item != 0;
  g->parallel = parallel != 0;
  g->share = share != 0;
  g->tile_div = tile_divisor;
  g->blocks_per_sm = blocks_per_sm;
  group_plan(g);
  return WADG_OK;
}

wadg_status wadg_group_info(const wadg_group* g, int32_t* nblocks, int32_t* threads,
                            int32_t* blocks_per_sm, int32_t* tile_divisor, int32_t* nitems,
                            int32_t* nvariants, int32_t* parallel, int32_t* share,
                            int32_t* nclusters, int32_t* per_item) {
  if (!g) return WADG_EINVAL;
  if (per_item) *per_item = g->per_item ? 1 : 0;
  if (nclusters) *nclusters = (int32_t)std::max<size_t>(1, g->cluster_of.size());
  if (nvariants) *nvariants = (int32_t)g->vars.size();
  if (parallel) *parallel = g->parallel ? 1 : 0;
  if (share) *share = g->share ? 1 : 0;
  if (nblocks) *nblocks = g->nblocks;
  if (threads) *threads = g->vars.empty() ? 0 : group_threads(g->vars[0].code);
  if (blocks_per_sm) *blocks_per_sm = g->blocks_per_sm;
  if (tile_divisor) *tile_divisor = g->tile_div;
  if (nitems) *nitems = (int32_t)g->items.size();
  return WADG_OK;
}

wadg_status wadg_group_run_steps(wadg_group* g, int64_t nsteps, const double* dt,
                                 double* const* probe_out) {
  if (!g) return WADG_EINVAL;
  wadg_status s0;
  if (!dt || nsteps < 0) return gfail(g, WADG_EINVAL, "bad arguments");
  for (size_t c = 0; c < g->ctx.size(); ++c)
    if (!(dt[c] > 0)) return gfail(g, WADG_EINVAL, "dt of member %d must be > 0", (int)c);
  if (nsteps == 0) return WADG_OK;
  if ((s0 = group_members_ready(g)) != WADG_OK) return s0;
  cudaSetDevice(g->device);
  // L2 clusters, each a group of its own with this group's tuning
  const auto cl = group_clusters(g);
  if (cl != g->cluster_of) {
    group_drop_clusters(g);
    for (const auto& c : cl) {
      std::vector<wadg_ctx*> m;
      for (int i : c) m.push_back(g->ctx[i]);
      wadg_group* sub = nullptr;
      s0 = wadg_group_create((int32_t)m.size(), m.data(), &sub);
      if (s0 != WADG_OK) {
        group_drop_clusters(g);
        return gfail(g, s0, "cluster set-up: %s", wadg_group_last_error(nullptr));
      }
      sub->stream = g->stream;
      g->clusters.push_back(sub);
    }
    g->cluster_of = cl;
  }
  if (!g->clusters.empty()) {
    for (size_t k = 0; k < g->clusters.size(); ++k) {
      wadg_group* sub = g->clusters[k];
      sub->tile_div = g->tile_div;
      sub->blocks_per_sm = g->blocks_per_sm;
      sub->parallel = g->parallel;
      sub->share = g->share;
      sub->per_item = g->per_item;
      std::vector<double> d;
      std::vector<double*> po;
      for (int i : g->cluster_of[k]) {
        d.push_back(dt[i]);
        po.push_back(probe_out ? probe_out[i] : nullptr);
      }
      s0 = wadg_group_run_steps(sub, nsteps, d.data(), po.data());
      if (s0 != WADG_OK) return gfail(g, s0, "%s", sub->err.c_str());
    }
    return WADG_OK;
  }
  const int64_t chunk = std::min<int64_t>(nsteps, 4096);
  for (wadg_ctx* x : g->ctx) {
    const size_t need = (size_t)chunk * x->nprobe * 6 * x->nb * 8;
    if (x->nprobe > 0 && x->pr_out.bytes < need) {
      invalidate_graphs(x);
      cudaError_t e = dalloc(x->pr_out, need);
      if (e != cudaSuccess) return gfail(g, WADG_ENOMEM, "probe records: %s", cudaGetErrorString(e));
    }
  }
  // the graphs of the last call still hold if no member changed since (same
  // generation and step) and every member's buffer parity moved alike;
  // otherwise rebuild the parameter tables and the graphs
  bool reuse = g->graph[0] && g->graph[1] && g->built_gen.size() == g->ctx.size();
  const int par0 = reuse ? (g->ctx[0]->cur ^ g->built_cur[0]) : 0;
  for (size_t c = 0; reuse && c < g->ctx.size(); ++c) {
    const wadg_ctx* x = g->ctx[c];
    reuse = x->gen == g->built_gen[c] && dt[c] == g->built_dt[c] &&
            (x->cur ^ g->built_cur[c]) == par0;
  }
  if (!reuse) {
    group_plan(g);
    wadg_status s = group_upload(g, dt);
    if (s != WADG_OK) return s;
    s = group_capture(g, dt);
    if (s != WADG_OK) return s;
    g->built_gen.clear();
    g->built_dt.assign(dt, dt + g->ctx.size());
    g->built_cur.clear();
    for (const wadg_ctx* x : g->ctx) {
      g->built_gen.push_back(x->gen);
      g->built_cur.push_back(x->cur);
    }
  }
  int64_t done = 0;
  int par = reuse ? par0 : 0;
  while (done < nsteps) {
    const int64_t n = std::min(chunk, nsteps - done);
    for (size_t c = 0; c < g->ctx.size(); ++c) {
      wadg_ctx* x = g->ctx[c];
      const double tt = x->t + done * dt[c];
      GCK(cudaMemcpyAsync(x->tdev.p, &tt, 8, cudaMemcpyHostToDevice, g->stream));
      GCK(cudaMemsetAsync(x->stepdev.p, 0, 8, g->stream));
    }
    for (int64_t i = 0; i < n; ++i) {
      GCK(cudaGraphLaunch(g->graph[par], g->stream));
      par ^= 1;
    }
    for (size_t c = 0; c < g->ctx.size(); ++c) {
      wadg_ctx* x = g->ctx[c];
      const size_t rec = (size_t)x->nprobe * 6 * x->nb;
      if (probe_out && probe_out[c] && rec)
        GCK(cudaMemcpyAsync(probe_out[c] + (size_t)done * rec, x->pr_out.p, (size_t)n * rec * 8,
                            cudaMemcpyDeviceToHost, g->stream));
    }
    GCK(cudaStreamSynchronize(g->stream));
    done += n;
  }
  for (size_t c = 0; c < g->ctx.size(); ++c) {
    wadg_ctx* x = g->ctx[c];
    x->t += nsteps * dt[c];
    if (nsteps & 1) x->cur ^= 1;   // each step flips the buffers once
  }
  return WADG_OK;
}

const char* wadg_group_last_error(const wadg_group* g) {
  return g ? g->err.c_str() : g_err.c_str();
}

}  // extern "C"

namespace {

void group_drop_clusters(wadg_group* g) {
  for (wadg_group* sub : g->clusters) wadg_group_destroy(sub);
  g->clusters.clear();
  g->cluster_of.clear();
}

}  // namespace
