/*
 * wadg.h -- C ABI of the GB300 library for nodal discontinuous Galerkin
 * time-domain (DGTD) Maxwell solves on tetrahedra with a stretched-coordinate
 * perfectly matched layer (SC-PML) whose conductivity varies inside elements,
 * applied through the weight-adjusted approximation (WAA) of the PML mass
 * matrices (Chen, Ozakin, Ahmed, Bagci: "A memory-efficient implementation
 * of perfectly matched layer with smoothly-varying coefficients in
 * discontinuous Galerkin time-domain method", Section II).
 *
 * Conventions (all entry points):
 *  - Every call returns a wadg_status; nothing aborts or exits.  On failure
 *    wadg_last_error(ctx) holds a one-line message until the next call.
 *  - Caller arrays are borrowed for the duration of the call and copied;
 *    the library keeps no caller pointer.
 *  - All device work is issued on the CUDA stream given to wadg_create (the
 *    legacy default stream when NULL).  Calls that return host data
 *    synchronise that stream first.
 *  - Element ids in and out of the library are the caller's (the row of
 *    etov); the internal reordering (PML class, then space-filling-curve
 *    order) is hidden.
 *  - Within an element, nodal values follow the equispaced node order:
 *    node (i,j,k), i+j+k <= N, at reference coordinates
 *    (r,s,t) = (-1 + 2i/N, -1 + 2j/N, -1 + 2k/N), enumerated with k
 *    outermost, then j, then i; the reference tetrahedron has vertices
 *    v1=(-1,-1,-1), v2=(1,-1,-1), v3=(-1,1,-1), v4=(-1,-1,1) mapped to the
 *    four vertices of the element in etov order.
 *  - Units are normalised: the background has eps = mu = 1 (so c0 = 1) and
 *    eps0 of the PML profile is a parameter (1 in normalised units).
 *  - A set-up call (wadg_set_mesh, wadg_set_materials, wadg_set_pml_profile,
 *    wadg_set_quadrature, wadg_set_sources, wadg_set_probes) that fails
 *    part-way, for instance because an allocation was refused, leaves the
 *    tables it was rebuilding incomplete: until the failed call (or
 *    wadg_set_mesh) has been repeated successfully, every call that launches
 *    kernels or reads or writes the state returns WADG_ESTATE without
 *    touching the device.  A failed wadg_set_sources / wadg_set_probes
 *    removes the previous sources / probes.
 */
#ifndef WADG_H
#define WADG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wadg_ctx wadg_ctx; /* opaque, owned by the library */

typedef enum {
  WADG_OK = 0,
  WADG_EINVAL = 1,       /* bad argument, malformed mesh, unsupported size */
  WADG_ENOMEM = 2,       /* a device or host allocation failed */
  WADG_ECUDA = 3,        /* a CUDA runtime call failed */
  WADG_ESTATE = 4,       /* call out of order (e.g. stepping before set_mesh) */
  WADG_ENOTFOUND = 5,    /* a source or probe point lies outside the mesh */
  WADG_ETIMEOUT = 6,     /* a bounded device-side wait gave up */
  WADG_ENONFINITE = 7,   /* the state holds NaN or Inf after stepping */
  WADG_EUNSUPPORTED = 8  /* valid request that this build does not provide */
} wadg_status;

/* Arithmetic of the stage kernels.  FP64: fields, operators and coefficients
 * in double.  FP32: fields, operators, coefficient samples in float; the
 * geometric factors stay double on the device and the source waveform, the
 * coefficient sampling and the objective sums are evaluated in double.
 * TF32 / BF16 (kappa = 1): as FP32, with the reference-operator
 * contractions (D_r, D_s, D_t, LIFT, V_q, P_q) on the tensor cores, operands
 * rounded to TF32 or BF16 (nearest) and accumulated in FP32. */
typedef enum { WADG_FP64 = 0, WADG_FP32 = 1, WADG_TF32 = 2, WADG_BF16 = 3 } wadg_precision;

/* PML implementation.
 *   WAA     eqs. 26-29, the weight-adjusted terms with the coefficients
 *           sampled at the volume quadrature nodes (the paper's method).
 *   STORED  eqs. 10-13 with per-element weighted mass matrices (eq. 15):
 *           the library stores M_k^-1 M_k^{b_u}, M_k^-1 M_k^{c_u} and
 *           M_k^-1 M_k^{d_u} per PML element and axis, and with kappa_max != 1
 *           also M_k^-1 M_k^{1/kappa_u} and (M_k^{a_u})^-1 M_k (15 N_p^2
 *           values, the paper's count; with kappa = 1 the last two are the
 *           identity and 9 N_p^2 are stored), built in double by a Stroud
 *           rule with N + 6 points per direction, (M^a)^-1 M_k by Gauss-Jordan
 *           elimination in double.  The reference "exact" scheme the WAA
 *           approximates; CUDA-core kernels in every precision (a TF32/BF16
 *           context runs its PML class on the FP32 CUDA-core kernel).
 *   EC      the WAA kernels with element-constant coefficients: every
 *           quadrature node of an element takes the profile's value at the
 *           element centroid (the piecewise-constant paving the paper
 *           compares against; for element-constant coefficients the WAA and
 *           stored schemes coincide, eq. 18). */
typedef enum { WADG_PML_WAA = 0, WADG_PML_STORED = 1, WADG_PML_EC = 2 } wadg_pml_scheme;

/* Stretching profiles of Section III, per axis u in {x, y, z}:
 *   d = max(0, (|u| - u0[u]) / L[u]),
 *   sigma_u = sigma_max[u] * d^p_sigma[u],
 *   kappa_u = 1 + (kappa_max[u] - 1) * d^p_sigma[u],
 * entering s_u = kappa_u + sigma_u / (j w eps0) (eq. 4) and the CPML tensors
 * a, b, c, d, kappa of eq. 9. */
typedef struct {
  double u0[3], L[3], sigma_max[3], p_sigma[3], kappa_max[3];
  double eps0;
} wadg_pml_profile;

/* Point electric dipole of moment amplitude * G(t) along unit vector dir at
 * point x, G(t) = exp(-(t - t0)^2 / (4 width^2)) (Section III's base-band
 * Gaussian pulse, with the minus sign the printed formula lacks); it drives
 * the current J = amplitude * G'(t) * dir * delta(x - x_s) in excitation
 * `batch` (0 <= batch < n_batch). */
typedef struct {
  double x[3], dir[3], t0, width, amplitude;
  int32_t batch;
} wadg_dipole;

/* Create a context for polynomial order N (1..5; the nodal basis of degree
 * N on each tetrahedron of Section II.A, N_p = (N+1)(N+2)(N+3)/6 nodes, the
 * orders p = 1..5 of Table I) with n_batch independent excitations advanced
 * together on CUDA device `device`, issuing work on
 * `cuda_stream` (a cudaStream_t, may be NULL).  EINVAL on bad N, precision
 * or n_batch (a TF32 context at N = 5 needs a compact volume rule before
 * it takes a PML, see wadg_set_quadrature); ECUDA if the device cannot be
 * used. */
wadg_status wadg_create(int N, wadg_precision prec, int32_t n_batch, int device,
                        void* cuda_stream, wadg_ctx** out);

/* Release every host and device resource of ctx (NULL is accepted). */
wadg_status wadg_destroy(wadg_ctx* ctx);

/* Mesh: nv vertices vxyz[nv][3] (double) and K tetrahedra etov[K][4]
 * (int64, 0-based).  The library computes in double the affine maps, J_k,
 * the metric terms, normals and surface Jacobians (Section II.A: straight-
 * sided elements, M_k = J_k M) and the face connectivity; faces with no
 * neighbour carry the perfect-electric-conductor condition.  EINVAL for an
 * index out of range, a non-positive Jacobian, or a face shared by more than
 * two elements.  Resets materials, PML, sources, probes and the state. */
wadg_status wadg_set_mesh(wadg_ctx* ctx, int64_t nv, const double* vxyz, int64_t K,
                          const int64_t* etov);

/* wadg_set_mesh with periodic boundaries: vcanon[nv] maps every vertex to a
 * representative (0 <= vcanon[v] < nv); two faces whose vertices have the same
 * representatives are neighbours, with their face nodes matched through that
 * vertex correspondence (so the two faces must be translates of each other
 * with the corresponding vertices in corresponding positions).  Used for the
 * lateral boundaries of the normal-incidence plane-wave box (Section III).
 * vcanon = NULL is wadg_set_mesh.  EINVAL as wadg_set_mesh, and for a
 * representative out of range. */
wadg_status wadg_set_mesh_periodic(wadg_ctx* ctx, int64_t nv, const double* vxyz, int64_t K,
                                   const int64_t* etov, const int64_t* vcanon);

/* Per-element relative permittivity and permeability eps_r[K], mu_r[K]
 * (caller element order, must be > 0); NULL means 1.  Enters the update
 * equations as eps_k, mu_k (eqs. 10, 11) and the upwind flux impedances. */
wadg_status wadg_set_materials(wadg_ctx* ctx, const double* eps_r, const double* mu_r);

/* PML profile (eq. 4 with the profiles of Section III).  An element belongs
 * to the PML class when any of its vertices has |u| > u0[u] on an axis whose
 * profile is active (sigma_max > 0 or kappa_max != 1); only PML elements
 * carry P^E, P^H.  The coefficients are sampled in double at the volume
 * quadrature nodes of each PML element (eq. 20 samples alpha_k(r_q)) and
 * stored per element as sigma_u (and kappa_u when kappa_max != 1); the
 * stored-matrix scheme holds its operators instead (see wadg_pml_scheme).
 * Pass NULL to remove the PML.  EINVAL for an unknown scheme, EUNSUPPORTED
 * for kappa_max != 1 with the weight-adjusted or element-constant scheme in a
 * TF32/BF16 context.  Resets the state and re-maps sources and probes. */
wadg_status wadg_set_pml_profile(wadg_ctx* ctx, const wadg_pml_profile* prof,
                                 wadg_pml_scheme scheme);

/* Volume quadrature of the weight-adjusted PML terms (eqs. 20, 21 and
 * 26-29: the coefficients are sampled at these points, V_q interpolates to
 * them and P_q = M^-1 V_q^T W projects back).  rstw[nq][4] holds the points
 * (r, s, t) on the reference tetrahedron and their weights w (summing to its
 * volume 4/3).  Section III uses rules of degree 2p with far fewer points
 * than the default, the conical-product (Stroud) rule of (N+1)^3 points
 * (degree 2N+1), which rstw = NULL restores.  The rule must have positive
 * weights, points inside the tetrahedron and integrate degree 2N exactly
 * (checked: P_q V_q must be the identity to 1e-10), else EINVAL.  The PML
 * kernels are compiled for two capacities: compact rules of at most
 * C_N = 4, 14, 24, 48, 84 points (N = 1..5) and rules of at most (N+1)^3
 * points; a rule is padded with zero-weight points to the capacity it falls
 * in (EUNSUPPORTED above (N+1)^3).  TF32 contexts at N = 5 need a compact
 * rule before a weight-adjusted or element-constant PML can be set; groups
 * take members with the default rule only.  The stored-matrix scheme keeps
 * its own rule.  Rebuilds the per-element tables when a mesh is set (as
 * wadg_set_pml_profile does: the state is reset, sources and probes are
 * re-mapped). */
wadg_status wadg_set_quadrature(wadg_ctx* ctx, int32_t nq, const double* rstw);

/* n point dipoles (copied).  ENOTFOUND if a point lies outside the mesh,
 * EINVAL for a batch index out of range or a non-positive width.  A point on
 * a shared face or vertex belongs to the lowest caller element id whose
 * barycentric coordinates are all >= -1e-12. */
wadg_status wadg_set_sources(wadg_ctx* ctx, int32_t n, const wadg_dipole* src);

/* n probe points xyz[n][3]; E and H there (the nodal expansion of
 * Section II.A evaluated at the point) are recorded after every full time
 * step by wadg_run_steps, as the field samples from which Section III
 * measures the PML reflection.  ENOTFOUND if a point is outside the mesh. */
wadg_status wadg_set_probes(wadg_ctx* ctx, int32_t n, const double* xyz);

/* State exchange.  The semi-discrete unknowns of Section II.A (the nodal
 * values of E, H and, in PML elements, the auxiliary fields P^E, P^H of
 * eqs. 5-8 that eqs. 10, 11 and 26-29 advance) as
 * q[n_batch][K][12][Np] (double) with the 12 components (Ex,Ey,Ez,Hx,Hy,Hz,
 * PEx,PEy,PEz,PHx,PHy,PHz), caller element order.  set_state ignores the P
 * components of non-PML elements (they are not stored) and sets the solution
 * time to t; get_state writes zeros there.  q == NULL in set_state zeros the
 * state.  set_state also clears the Runge-Kutta register and the probe
 * objective.
 * on_device = 0: q is host memory; the call converts on the host and copies
 * (synchronising the context's stream).
 * on_device = 1: q is device memory on the context's device; a kernel on
 * the context's stream converts between q and the internal blocks, with no
 * host copy, and the call returns without waiting (q must stay valid until
 * the stream has passed the exchange, as for any stream-ordered work). */
wadg_status wadg_set_state(wadg_ctx* ctx, const void* q, double t, int on_device);
wadg_status wadg_get_state(wadg_ctx* ctx, void* q, double* t, int on_device);

/* Device bytes the state buffers of the current mesh and PML need
 * (the two E,H copies, their register, P and its register; each block
 * padded and 256-byte aligned): the size wadg_bind_state wants.  ESTATE
 * without a mesh. */
wadg_status wadg_state_bytes(const wadg_ctx* ctx, size_t* bytes);

/* Place the state buffers in caller-owned device memory dev (on the
 * context's device, 256-byte aligned, at least wadg_state_bytes bytes), for
 * callers such as PyTorch whose allocator owns the device memory.  The
 * current state moves into dev (device to device) and the library releases
 * its own buffers.  dev must stay allocated until the context is destroyed
 * or the state is unbound with dev = NULL (the library then allocates its
 * own buffers again and moves the state back).  Later set-up calls that
 * rebuild the state (wadg_set_mesh, wadg_set_pml_profile, ...) keep using
 * dev, and fail with EINVAL when it is too small for the new state.  Bound
 * bytes do not count against wadg_set_memory_limit.  The internal layout of
 * dev is the library's; exchange values through wadg_set_state /
 * wadg_get_state. */
wadg_status wadg_bind_state(wadg_ctx* ctx, void* dev, size_t bytes);

/* Bytes the context has copied from host to device and back since it was
 * created: state exchanges through host memory, probe records, objective
 * reads and the few bytes of step clocks and status flags. */
wadg_status wadg_transfer_bytes(const wadg_ctx* ctx, size_t* h2d, size_t* d2h);

/* One stage i (0..4) of the five-stage fourth-order low-storage Runge-Kutta
 * scheme: res <- A_i res + dt * f(q, t + c_i dt); q <- q + B_i res, where f
 * is the semi-discrete right-hand side (the curl with upwind flux of the
 * equation after eq. 15, and eqs. 26-29 in PML elements).  Does not change
 * the solution time held by the context. */
wadg_status wadg_rk_stage(wadg_ctx* ctx, int stage, double t, double dt);

/* Advance every excitation by nsteps full steps of size dt from the current
 * solution time: the explicit time marching of the semi-discrete system
 * (Section II.B), each step the five stages of wadg_rk_stage.  If probe_out
 * is not NULL it receives
 * probe_out[nsteps][nprobe][6][n_batch] (double; Ex..Hz after each step).
 * The FP64 objective sum over probes and steps of |E|^2 accumulates per
 * excitation (wadg_objective).  ENONFINITE if the state became non-finite. */
wadg_status wadg_run_steps(wadg_ctx* ctx, int64_t nsteps, double dt, double* probe_out);

/* Measurement aid: run `reps` eager Runge-Kutta stages (stage index cycling
 * 0..4, time = current solution time) and return in ms_out[2] the average
 * device duration of one launch of the non-PML stage kernel (ms_out[0]) and
 * of the PML stage kernel (ms_out[1]), timed with CUDA events on the
 * context's stream.  Advances the state like wadg_rk_stage. */
wadg_status wadg_profile_stage(wadg_ctx* ctx, int reps, double dt, double* ms_out);

/* Gradient of the probe objective J_b = sum over the nsteps steps and the
 * probes of |E(x_p)|^2 (excitation b, FP64 sums) with respect to the
 * per-element relative permittivity eps_r and, per axis, the PML parameters
 * sigma_max and p_sigma (profiles of Section III with kappa = 1, so eq. 9 has
 * a = 1), by the discrete adjoint of the Runge-Kutta recursion and of the
 * semi-discrete operator (upwind flux, eqs. 26-29).  Starts from the current
 * state and time; the forward pass stores a checkpoint every ckpt_every
 * steps and the reverse pass recomputes each segment from its checkpoint,
 * keeping the input of every stage of the segment, then runs the segment's
 * reverse stages on them.  On return the state is the forward state after nsteps steps (as after
 * wadg_run_steps).  Outputs (any may be NULL): J_out[n_batch],
 * dJ_deps[n_batch][K] (caller element order), dJ_dsigma_max[n_batch][3],
 * dJ_dp_sigma[n_batch][3].  EUNSUPPORTED for the TF32 and BF16 precisions,
 * kappa_max != 1 or a PML scheme other than WADG_PML_WAA; ESTATE without
 * probes.  Device memory: about
 * (nsteps/ckpt_every + 5 min(ckpt_every, nsteps) + 6) copies of the state. */
wadg_status wadg_adjoint(wadg_ctx* ctx, int64_t nsteps, double dt, int32_t ckpt_every,
                         double* J_out, double* dJ_deps, double* dJ_dsigma_max,
                         double* dJ_dp_sigma);

/* wadg_run_steps for callers that cannot allocate device memory when they
 * step: for example code that runs under a fixed device-memory budget handed
 * to it by an enclosing application, or a caller that must not trigger the
 * implicit device synchronisation an allocation can bring.  (The paper has
 * no counterpart; this is a property of the library, not of the method.)
 * Same arguments, results and errors as wadg_run_steps, but this call
 * allocates nothing: it launches the stage kernels directly instead of
 * replaying a captured graph, and its scratch -- the device time and step
 * counters, the non-finite flag and the probe records of a chunk of steps on
 * their way to probe_out -- lives in one fixed 16 MiB device array of the
 * library (held on every GPU that loads the library until the process
 * exits).  Steps are processed in chunks whose probe records fit the array;
 * EINVAL if the records of a single step (nprobe * 6 * n_batch doubles) do
 * not fit.  Each call looks up the array's device address on the context's
 * device (cudaGetSymbolAddress); with lazy module loading the first call on
 * a device also loads the module, so it should come before any stream
 * capture.  Every call shares the one array per device and sets the counters
 * it needs before use, so calls whose work overlaps on the GPU (other
 * threads, other streams) race on it. */
wadg_status wadg_run_steps_noalloc(wadg_ctx* ctx, int64_t nsteps, double dt, double* probe_out);

/* Largest step for the given CFL number of the explicit time marching
 * (Section II.B; the paper states no step rule, this is the usual nodal DG
 * bound): dt = cfl * 2 / ((N+1)^2 * max_{k,f} Fscale_{k,f}), Fscale = sJ/J. */
wadg_status wadg_stable_dt(const wadg_ctx* ctx, double cfl, double* dt_out);

/* Objective J_b = sum over probes and recorded steps of |E|^2 for each
 * excitation b: J_out[n_batch]. */
wadg_status wadg_objective(wadg_ctx* ctx, double* J_out);

/* Device bytes held for the field state (q, res and the P fields), for the
 * per-element PML coefficients (the samples of the weight-adjusted and
 * element-constant schemes, the operators of the stored-matrix scheme), for
 * the reference operators, and for the per-element geometry and
 * connectivity: the memory comparison of Section II.B (15 N_p^2 values per
 * PML element for stored matrices against samples at N_q points for the
 * weight-adjusted scheme) and Table I.  Any pointer may be NULL. */
wadg_status wadg_memory_report(const wadg_ctx* ctx, size_t* bytes_state,
                               size_t* bytes_pml_coeff, size_t* bytes_operators,
                               size_t* bytes_geometry);

/* Mesh sizes after set_mesh / set_pml_profile: elements, PML elements,
 * nodes per element, volume quadrature nodes per element (of the rule, not
 * counting the padding to the kernels' capacity). */
wadg_status wadg_mesh_info(const wadg_ctx* ctx, int64_t* K, int64_t* K_pml, int32_t* Np,
                           int32_t* Nq);

/* Block until all work issued by ctx has finished. */
wadg_status wadg_synchronize(wadg_ctx* ctx);

/* Cap on the device bytes this context may hold (0, the default: no cap).
 * Every device buffer the library allocates for the context counts: state,
 * geometry, coefficients, operators, probe records, adjoint buffers.  A
 * request that would take the context past the cap fails before any device
 * call, as an exhausted device would: the call returns WADG_ENOMEM and the
 * context stays usable (raise the cap and repeat the call).  A cap below
 * what is already held blocks further allocations only.  held_out (may be
 * NULL) receives the bytes the context holds now.  Allocations of a group
 * (wadg_group_*) do not count.  (The paper has no counterpart.) */
wadg_status wadg_set_memory_limit(wadg_ctx* ctx, size_t bytes, size_t* held_out);

/* Failure-detection test aid for the TF32 and BF16 contexts, the ones whose
 * kernels wait on device-side signals (the mbarriers between the tensor-core
 * issuing thread and the compute warps).  Every such wait gives up after
 * about one second, sets the context's error flag and lets the kernel drain
 * the products it issued, release its tensor memory and end; the call that
 * launched it (wadg_rk_stage, wadg_run_steps, wadg_run_steps_noalloc) then
 * returns WADG_ETIMEOUT, with the state partly updated.  This call arms one
 * request: the first block of a later tensor-core stage launch that takes it
 * issues the flux product of its first tile without the completion signal,
 * so that one wait runs out.  Nothing faults, traps or waits without limit,
 * and the context stays usable (set the state again and step).  The request
 * stays armed until a launch takes it.  EUNSUPPORTED for FP64 and FP32
 * contexts.  (The paper has no counterpart; this tests the library's error
 * path.) */
wadg_status wadg_arm_wait_timeout(wadg_ctx* ctx);

/* Measured fused multiply-add throughput of device `device`'s CUDA cores in
 * TFLOP/s (2 flops per FMA): FP64 (fp64 != 0) or FP32, from independent
 * register FMA chains in every thread of 4 blocks per SM, timed with CUDA
 * events.  The roofline denominator of the FP64 and FP32 CUDA-core stage
 * kernels.  (The paper has no counterpart; this is a measurement aid.) */
wadg_status wadg_fma_peak(int device, int fp64, double* tflops);

/* Reference-element operator of order N (host only, no device needed), for
 * checking the library's set-up against an independent construction.
 * which: 0 Dr, 1 Ds, 2 Dt ([Np][Np]), 3 LIFT ([Np][4 Nfp]), 4 V_q ([Nq][Np]),
 * 5 P_q ([Np][Nq]), 6 quadrature nodes and weights ([Nq][4] = r,s,t,w),
 * 7 M^{-1} ([Np][Np]).  `cap` is the capacity of out in doubles; *n_out
 * receives the count.  EINVAL for a bad N or which, or a too small cap. */
wadg_status wadg_reference_operator(int N, int which, double* out, int64_t cap,
                                    int64_t* n_out);

/* Message of the last failed call on ctx (or of the last failed
 * wadg_create / wadg_reference_operator when ctx is NULL). */
const char* wadg_last_error(const wadg_ctx* ctx);

/* ---------------------------------------------------------------- groups
 * Several contexts advanced together (the batching form: meshes of uneven
 * size, order and precision).  A Runge-Kutta stage of the whole group is one
 * of two launch patterns, chosen by wadg_group_autotune or fixed by
 * wadg_group_set_tuning:
 *  - grouped variant kernels: one launch per variant (order N, element class)
 *    present, of a CUDA-core kernel compiled for that variant alone, whose
 *    blocks start on the variant's (member, class) items in proportion to
 *    their algorithmic flops and then take tiles from per-item counters until
 *    none are left.  Only for FP32 members (WADG_FP32) with the (N+1)^3 rule
 *    and the weight-adjusted or element-constant PML;
 *  - per-item launches: every (member, class) item as the member's own stage
 *    kernel (any precision, volume rule and PML scheme: tensor-core members
 *    included).  A group with any member outside the first kind uses this.
 * The launches of a stage run in turn or on parallel branches, so the SMs one
 * launch leaves at its tail go to the others.  One step (the stage launches
 * and each member's probe and clock kernels) is captured in a CUDA graph.
 * Each member advances exactly as wadg_run_steps advances it (the stage of
 * eqs. 10, 11 and 26-29 with the time marching of Section II.B), bit for bit;
 * the grouping itself has no counterpart in the paper.  Members: contexts
 * with a mesh on one device; the group runs on the first member's stream.
 * Each member keeps its own state, time, probes and records.  The group
 * refers to its members: destroy the group before any member. */
typedef struct wadg_group wadg_group;

/* EINVAL for a null or repeated member or members on different devices,
 * ESTATE for a member without a mesh or with an incomplete set-up. */
wadg_status wadg_group_create(int32_t n, wadg_ctx* const* ctxs, wadg_group** out);
wadg_status wadg_group_destroy(wadg_group* g);

/* Tile sizes and grid: times `reps` grouped stage launches for every
 * candidate (grouped variant kernels, or every (member, class) item launched
 * as its single-context kernel; elements per tile = the largest that fits /
 * {1, 2, 4}; 1..4 blocks per SM within each variant's occupancy limit; a
 * stage's launches on parallel branches or one after the other; each
 * variant's grid the whole GPU or its share by algorithmic flops; each
 * variant keeps the block shape of its single-context kernel) with
 * the members' step sizes
 * dt[n], keeps the fastest and writes its time per stage launch (ms) to
 * ms_out (may be NULL).  The stages run on the members' current state, which
 * is left undefined: call it before wadg_set_state. */
wadg_status wadg_group_autotune(wadg_group* g, const double* dt, int32_t reps, double* ms_out);

/* Set the launch shape without timing (the values wadg_group_autotune
 * chooses among): per_item (1: every item as its single-context kernel),
 * parallel (1: a stage's launches on parallel branches), share (1: each
 * variant's grid its share of the GPU), tile_divisor (1..64), blocks_per_sm
 * (1..8, capped by each variant's occupancy).  EINVAL out of range;
 * EUNSUPPORTED for per_item = 0 in a group whose members the grouped variant
 * kernels do not serve. */
wadg_status wadg_group_set_tuning(wadg_group* g, int32_t per_item, int32_t parallel,
                                  int32_t share, int32_t tile_divisor, int32_t blocks_per_sm);

/* The current launch shape: total blocks (all variants), threads per block
 * of the heaviest variant, blocks per SM (each variant is capped by its own
 * occupancy), tile divisor, work items, variants (launches per stage),
 * whether a stage's variant launches run on parallel branches (1) or in turn
 * (0), and whether each variant's grid is its share of the GPU (1) or the
 * whole GPU (0), the number of L2 clusters of the last wadg_group_run_steps (1: all
 * members advanced together), and whether each item is launched as its
 * single-context kernel (1) instead of the grouped variant kernels (0).  Any
 * pointer may be NULL. */
wadg_status wadg_group_info(const wadg_group* g, int32_t* nblocks, int32_t* threads,
                            int32_t* blocks_per_sm, int32_t* tile_divisor, int32_t* nitems,
                            int32_t* nvariants, int32_t* parallel, int32_t* share,
                            int32_t* nclusters, int32_t* per_item);

/* nsteps steps of every member with its own dt[n]; probe_out[n] (entries may
 * be NULL, or probe_out itself) receive each member's records laid out as in
 * wadg_run_steps.  Gives each member the values wadg_run_steps would.  The
 * members are packed into clusters whose per-step device data fits half of
 * the L2 (members above that form one cluster); each cluster runs all nsteps
 * before the next, so small members step out of L2. */
wadg_status wadg_group_run_steps(wadg_group* g, int64_t nsteps, const double* dt,
                                 double* const* probe_out);

/* Text of the last error of a group call (of the creating call for a NULL
 * group). */
const char* wadg_group_last_error(const wadg_group* g);

#ifdef __cplusplus
}
#endif
#endif /* WADG_H */
