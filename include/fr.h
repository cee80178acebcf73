/*
 * libfr -- GB300 (sm_103a) Flux Reconstruction LES residual, RK4 update,
 * wall forces, FW-H data-surface sampling and FW-H integration.
 *
 * The operations follow Hamedi & Vermeire, "Far-Field Aeroacoustic Shape
 * Optimization Using Large Eddy Simulation" (arXiv 2501.05709):
 *   - compressible Navier-Stokes in conservation form, Section 2.1, Eqs. 1-7;
 *   - Flux Reconstruction on curved hexahedra with implicit LES, Section 1,
 *     Section 2.1, Section 3.1;
 *   - mean lift/drag, Section 3.2 (Table 1) and Eq. 8;
 *   - data-surface sampling of rho, p, velocity, Section 3.1 and 3.4;
 *   - FW-H moving-medium integration with spanwise duplication, Appendix B
 *     (Eqs. B.1-B.14) and Section 3.3.1;
 *   - Welch power spectral density of the observer pressure, Section 3.3;
 *   - the energy source of the monopole validation cases, Appendix D
 *     (Eq. D.1);
 *   - adaptive time-step size, Section 3.1 (the integrator stays RK4);
 *   - variable polynomial order by element (the sponge zones of
 *     Section 3.1).
 * FR details the paper leaves open are fixed as: Gauss-Legendre solution and
 * flux points, DG or Huynh-g2 correction functions, Rusanov inviscid flux,
 * BR2 viscous flux, classic four-stage RK4.
 *
 * Conventions for every call:
 *   - return value: FR_OK (0) or a negative FR_E* code; fr_last_error()
 *     gives a message for the calling thread.
 *   - host arrays passed in are read during the call and never retained;
 *   - device pointers passed in belong to the caller, are used in stream
 *     order on the given cudaStream_t (passed as void*; NULL = legacy default
 *     stream) and are never freed by the library;
 *   - the library owns its internal device buffers (freed by fr_destroy);
 *   - there is no CPU fallback: every compute call runs CUDA kernels and
 *     fails with FR_ECUDA when no usable GPU is present.
 *
 * Canonical state layout: [E][nvar][Nsp], E elements (all candidates
 * concatenated in load order), nvar = dim + 2 conserved variables
 * (rho, rho*V_1..V_dim, rho*E), Nsp = (p+1)^dim solution points with index
 * i_0 + (p+1) i_1 (+ (p+1)^2 i_2), i_0 along xi_1 fastest.
 */
#ifndef LIBFR_FR_H
#define LIBFR_FR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FR_OK 0
#define FR_EINVAL -1     /* bad argument */
#define FR_ENOMEM -2     /* device or host allocation failed */
#define FR_ECUDA -3      /* CUDA runtime error (no device, launch failure) */
#define FR_ENONFINITE -4 /* NaN or Inf found in the state */
#define FR_ETIMEOUT -5   /* a bounded device wait expired */
#define FR_EWINDOW -6    /* FW-H: the unified observer window is empty */
#define FR_EMESH -7      /* invalid geometry or connectivity */

#define FR_FP64 0        /* all state and arithmetic in double */
#define FR_FP32 1        /* state and arithmetic in float; metrics computed in
                            double and rounded once; force, energy and FW-H
                            accumulators in double */
#define FR_TF32_TC 2     /* FR_FP32 with the gradient and divergence line
                            operators of the residual on the tensor cores,
                            operands rounded to TF32, FP32 accumulation
                            (3D, p = 3 or 4) */
#define FR_BF16X3_TC 3   /* as FR_TF32_TC with each operand split into two
                            bfloat16 parts (hi + lo) and three products
                            (hi hi + hi lo + lo hi), FP32 accumulation */

#define FR_CORR_DG 0       /* g_L = right Radau polynomial of degree p+1 */
#define FR_CORR_HUYNH_G2 1 /* Huynh's g2 */

#define FR_BC_WALL 1      /* no-slip adiabatic wall (slip wall when inviscid) */
#define FR_BC_FARFIELD 2  /* characteristic (Riemann-invariant) far field */

typedef struct fr_ctx fr_ctx;

/* One mesh (one candidate).  nodes: [nelem][(q+1)^dim][dim] double, nodes at
 * the equispaced reference points of each direction, local index
 * a + (q+1) b (+ (q+1)^2 c).  conn: [nelem][2 dim][3] int32; face 2d is
 * xi_d = -1, face 2d+1 is xi_d = +1; an interior face holds (neighbour
 * element, neighbour face, orientation) with the orientation code of the face
 * point map (dim 2: bit 0 reverses; dim 3: bit 2 swaps the two face indices,
 * then bit 0 / bit 1 reverse the first / second); a boundary face holds
 * (-FR_BC_WALL or -FR_BC_FARFIELD, 0, 0).  Element numbers are local to the
 * candidate. */
typedef struct {
    int dim;
    int nelem;
    int geom_order;
    const double* nodes;
    const int32_t* conn;
} fr_mesh_desc;

typedef struct {
    int order;          /* p, 1..4 */
    int correction;     /* FR_CORR_* */
    int precision;      /* FR_FP64, FR_FP32, FR_TF32_TC or FR_BF16X3_TC */
    int viscous;        /* 0: Euler, 1: Navier-Stokes (BR2) */
    double gamma;       /* ratio of specific heats (1.4 in Section 2.1) */
    double prandtl;     /* Pr (0.71 in Section 2.1) */
    double mu;          /* constant dynamic viscosity */
    double br2_eta;     /* BR2 lifting penalty (1.0 default) */
    double rho_inf;     /* free stream: far-field state, force scale, */
    double p_inf;       /*   sampled-deviation reference               */
    double vel_inf[3];
    double dt;          /* RK4 time step */
    double lift_dir[3]; /* unit vectors for C_L / C_D */
    double drag_dir[3];
    double ref_area;    /* chord * span; C = F / (1/2 rho_inf |V_inf|^2 ref_area) */
} fr_options;

/* Context sizes: out[0]=dim, [1]=order p, [2]=nvar, [3]=Nsp, [4]=total
 * elements E, [5]=ncand, [6]=precision, [7]=metric path: 0 per-point metrics
 * (some element is curved), 1 every element affine (one metric set per
 * element), 2 every element affine and axis-aligned (diagonal metrics). */
int fr_ctx_dims(const fr_ctx* ctx, int64_t out[8]);

/* fr_mesh_load (Section 3.1 mesh of curved hexahedra; FR set-up of Section 1):
 * builds reference operators, curved-element metric terms in
 * conservative-curl form, shared face normals and the face-pair table for
 * ncand meshes (m[0..ncand-1]) concatenated into one batch, uploads them and
 * allocates the state.  Errors: FR_EINVAL (bad sizes or options), FR_EMESH
 * (non-positive Jacobian, asymmetric or mismatched connectivity), FR_ENOMEM,
 * FR_ECUDA.  *out is set to NULL on error. */
int fr_mesh_load(const fr_mesh_desc* m, int ncand, const fr_options* o, fr_ctx** out);

/* Releases every device and host resource of ctx (NULL is accepted). */
int fr_destroy(fr_ctx* ctx);

/* Message of the last error raised on this thread ("" if none). */
const char* fr_last_error(void);

/* Physical solution-point coordinates, host double [E][Nsp][dim], for cand
 * (or all candidates when cand < 0).  The caller owns xyz. */
int fr_sp_coords(const fr_ctx* ctx, int cand, double* xyz);

/* Element offset and count of candidate cand within the batch. */
int fr_cand_range(const fr_ctx* ctx, int cand, int64_t* first, int64_t* count);

/* State upload / download in the canonical layout as double.  cand < 0
 * addresses the whole batch.  on_device != 0: u is a device pointer.
 * fr_state_set also resets the RK stage buffers, projects elements of
 * reduced degree (fr_set_element_order) and clears the addressed candidates'
 * non-finite flags (fr_nonfinite).  fr_state_get copies the state and then
 * returns FR_ENONFINITE when an addressed candidate's flag is set (or, for a
 * host copy, when a copied value is NaN or Inf).  Both calls synchronise the
 * given stream before returning.  A host array that the CUDA runtime has
 * page-locked and mapped (cudaHostAlloc, cudaHostRegister, a pinned torch
 * tensor) is read or written in place by the conversion kernel over the
 * CPU-GPU link; pageable host memory goes through a device staging buffer
 * (allocated on first use, E * nvar * Nsp doubles, FR_ENOMEM if that fails).
 * Both give the same state bit for bit. */
int fr_state_set(fr_ctx* ctx, int cand, const double* u, int on_device, void* stream);
int fr_state_get(fr_ctx* ctx, int cand, double* u, int on_device, void* stream);

/* Non-finite detection on the device: the last stage of every step tests each
 * new state value (exponent bits all ones: NaN or infinity) and sets a flag
 * for the element's candidate, so one diverging candidate of a batch does not
 * hide behind the others.  *flag = 1 when candidate cand's flag (cand = -1:
 * any candidate's) is set, else 0.  Flags stay set until fr_state_set.
 * Synchronises the device.  Errors: FR_EINVAL. */
int fr_nonfinite(const fr_ctx* ctx, int cand, int* flag);

/* Explicit time integrator in coefficient form (Section 3.1 integrates with
 * an optimal explicit scheme whose coefficients are given in the work it
 * cites, not in the paper; this call takes any scheme that fits the form).
 * Stage i = 1..nstages of a step from u0 with input v (v = u0 at stage 1)
 * and k = R(v) at time t_n + tau_i dt:
 *   acc <- e_i acc + f_i dt k                    (acc = 0 before stage 1)
 *   v   <- a_i u0 + b_i v + c_i dt k + d_i acc   (rounded as ((a u0 + d acc)
 *                                                 + b v) + (c dt) k, one FMA
 *                                                 per step)
 * and the last v is the new state.  coef: host [nstages][6] doubles
 * (a, b, c, d, e, f).  This covers classic RK4 (stage i: (1,0,1/2,0,0,1/6),
 * (1,0,1/2,0,1,1/3), (1,0,1,0,1,1/3), (1,0,1/6,1,1,0), which reproduces the
 * built-in RK4 bit for bit), Shu-Osher SSP forms (d = e = f = 0) and 2N
 * low-storage forms (a = c = 0, b = 1).  The stage times tau_i (for the
 * energy source) are the scheme's own values on du/dt = 1.  nstages = 0
 * returns to the built-in RK4.  Forces and surface samples are taken at the
 * start of each step as before.  Errors: FR_EINVAL (nstages outside 0..16,
 * non-finite coefficients, or a scheme whose step on du/dt = 1 does not
 * advance u by dt), FR_ENOMEM (odd stage counts need a third trace buffer).
 * Rebuilds the step's CUDA graph on its next replay. */
int fr_set_rk_scheme(fr_ctx* ctx, int nstages, const double* coef);

/* fr_residual (Eq. 1 semi-discretised: du/dt = R(u)): one residual evaluation
 * of the whole batch.  u and R are device pointers in the context precision
 * (double for FR_FP64, float otherwise), canonical layout, E*nvar*Nsp
 * values each; they must not overlap.  Uses the context's trace buffers, so
 * calls on one context must not run concurrently. */
int fr_residual(fr_ctx* ctx, const void* u, void* R, void* stream);

/* fr_rk_step: advances the internal state by nsteps classic RK4 steps of
 * size dt (each step: 4 residual evaluations fused with the stage update;
 * fr_set_rk_scheme selects another explicit scheme),
 * accumulating the wall force every step and appending one record to every
 * registered FW-H surface every step.  Enqueued on stream; returns without
 * synchronising. */
int fr_rk_step(fr_ctx* ctx, int nsteps, void* stream);

/* Per-candidate time step (the batched MADS poll of Section 2.2 advances
 * candidates of uneven meshes together, each at its own stable step): every
 * element of candidate cand uses dt from now on (fr_options.dt until set).
 * Errors: FR_EINVAL (cand out of range, dt <= 0), FR_ENOMEM. */
int fr_set_cand_dt(fr_ctx* ctx, int cand, double dt);

/* Energy source of Appendix D (Eq. D.1 and its multi-monopole form): adds
 *   s(x, t) = sum_m A_m exp(-k_m |x - x_m|^2) sin(2 pi f_m t)
 * to the energy equation of candidate `cand`, evaluated at every solution
 * point at the stage time (classic RK4: t_n, t_n + dt/2, t_n + dt/2,
 * t_n + dt; fr_residual uses t_n).
 *   src   host, [nsrc][6] doubles (A, k, x, y, z, f) per source, copied;
 *         0 <= nsrc <= 4 (nsrc = 0 removes the candidate's sources); k >= 0;
 *         z ignored in 2D.  Elements whose weights exp(-k|x - x_m|^2) are all
 *         below 1e-30 are skipped.
 *   t0    the candidate's time t_n from now on; every RK4 step advances it by
 *         the candidate's dt (fr_set_cand_dt or the options' dt).
 * Errors: FR_EINVAL (bad candidate, nsrc, non-finite values, k < 0, a
 * candidate with elements of reduced degree, fr_set_element_order),
 * FR_ENOMEM.  Rebuilds the step's CUDA graph on its next replay. */
int fr_set_source(fr_ctx* ctx, int cand, int nsrc, const double* src, double t0);

/* The candidate's source time t_n (0 if no source was ever set). */
int fr_source_time(const fr_ctx* ctx, int cand, double* t);

/* Adaptive time step (Section 3.1 runs with adaptive time stepping; its
 * integrator's coefficients are in the cited work, not in the paper, so the
 * update stays classic RK4 and only the step size adapts).  With cfl > 0,
 * every RK4 step first sets each candidate's step from the state at the start
 * of the step:
 *   dt = cfl / max_e lambda_e,
 *   lambda_e = max_sp (|V| + c) (p+1)^2 / h_e + max_sp (mu / rho) (p+1)^4 / h_e^2
 * (the viscous term only with viscous physics), h_e = min over solution
 * points and directions d of 2 |J| / |S[d,:]|.  All on the device, so graph
 * replay adapts too.  cfl <= 0 returns to the fixed steps (fr_set_cand_dt or
 * the options' dt).  Forces keep per-step averages; surface samples are taken
 * every `every` steps whatever their spacing in time.
 * Errors: FR_EINVAL (non-finite cfl), FR_ENOMEM. */
int fr_set_adaptive_dt(fr_ctx* ctx, double cfl);

/* The candidate's current step (the last adaptive one, or the fixed one). */
int fr_cand_dt(const fr_ctx* ctx, int cand, double* dt);

/* Variable polynomial order (Section 3.1: the solution degree drops from the
 * context's p near the body to 0 in the outer rings, so that the coarse,
 * low-order far field absorbs outgoing waves).  order[i] in 0..p is the degree
 * of element i of candidate cand (cand = -1: of the whole batch, E entries);
 * order = NULL gives the candidate's elements p again.  An element of degree
 * q < p is a degree-q FR element on its own (q+1)^dim GL points, with the
 * degree-q operators (at q = 0 the one linear correction function) and its
 * metric terms taken as the degree-p interpolants evaluated at those points,
 * while every face keeps the degree-p flux points, so faces stay conforming:
 *   - its state is stored as the values of its degree-q polynomial at the
 *     degree-p points (the current state and every state set later are
 *     projected onto that space with the 1D L2 projection
 *     Pi_q[i][j] = sum_{k<=q} P_k(x_i) P_k(x_j) w_j (2k+1)/2 along each
 *     direction), so traces, sampling and state transfers are unchanged;
 *   - the jump u_c - u_f and the common normal flux at the degree-p face
 *     points reach it through the L2 projection onto degree q along each face
 *     direction (a mortar that keeps each face's mean);
 *   - its residual, computed at its q points, is evaluated at the degree-p
 *     points; its BR2 face gradients, built at its q face points, likewise.
 * With q = p this is the uniform scheme; the scheme stays conservative and
 * keeps a free stream on affine elements.  Reduced elements are handled by
 * their own kernels, so they cost degree-q work.  A candidate with an energy
 * source (fr_set_source) keeps a uniform degree.  Errors: FR_EINVAL (cand out
 * of range, an order outside 0..p, a candidate with a source), FR_ENOMEM.
 * Synchronises the device; rebuilds the step's CUDA graph on its next
 * replay. */
int fr_set_element_order(fr_ctx* ctx, int cand, const int32_t* order);

/* Same as fr_rk_step but replays a CUDA graph of one step (captured on first
 * use for the current surfaces and options).  Bit-identical results. */
int fr_rk_step_graph(fr_ctx* ctx, int nsteps, void* stream);

/* fr_forces (Section 3.2 mean lift and drag): out[0] = C_L and out[1] = C_D
 * of the last accumulated step, out[2] = mean C_L, out[3] = mean C_D over
 * the accumulated steps, out[4] = number of steps.  Synchronises the
 * context's work.  Returns FR_ENONFINITE (out still filled) when the
 * candidate's non-finite flag is set.  fr_forces_reset zeroes the running
 * means. */
int fr_forces(fr_ctx* ctx, int cand, double out[5]);
int fr_forces_reset(fr_ctx* ctx);

/* Volume integrals in double of the current state of candidate cand:
 * out[0..nvar-1] = integral of each conserved variable, out[nvar] = kinetic
 * energy integral (1/2 rho |V|^2).  Used for conservation checks and the
 * Taylor-Green kinetic-energy history. */
int fr_integrals(fr_ctx* ctx, int cand, double* out);

/* fwh_register (Section 3.1 permeable data surface; the paper collects every
 * 25 steps): locates npts physical points xyz (host double [npts][3]) in
 * candidate cand by Newton inversion of the element maps (lowest element id
 * wins on shared faces) and reserves a device history of capacity records.
 * fr_rk_step appends a record at the start of every `every`-th step (every
 * >= 1; the step counter is kept on the device, so graph replays stay in
 * phase).  *handle identifies the surface.  Errors: FR_EINVAL (point outside
 * the mesh, bad sizes), FR_ENOMEM. */
int fwh_register(fr_ctx* ctx, int cand, int npts, const double* xyz, int capacity, int every, int* handle);

/* fwh_sample: appends one record of (rho, V_1..V_3, p) at every point of
 * surface handle from the current state (FR_EINVAL when full).  Records are
 * stored as deviations from the free stream in the context precision. */
int fwh_sample(fr_ctx* ctx, int handle, void* stream);

/* Copies the records of surface handle to out (host double
 * [nrec][npts][5], total rho, V, p); *nrec gets the record count.  out may
 * be NULL to query the count.  fwh_clear empties the history. */
int fwh_history(fr_ctx* ctx, int handle, double* out, int* nrec);
int fwh_clear(fr_ctx* ctx, int handle);

/* fwh_integrate (Appendix B, Eqs. B.2-B.14, advanced-time approach, on the
 * data surface repeated ncopies times along z at spacing Lspan, Section
 * 3.3.1): acoustic pressure p'(t*) at each of nobs observers.
 * Device inputs (double): hist [nt][npts][5] = (rho, V_1, V_2, V_3, p) at
 * source times tau0 + k dtau; y [npts][3] panel centres; n [npts][3] outward
 * unit normals; dS [npts] panel areas.  Host inputs: obs [nobs][3],
 * Minf[3] (mean-flow Mach vector), c0, rho0, p0.  ncopies must be odd.
 * Output: p_out (device double [nobs][cap]) receives p'(t*_i) for
 * i < nt_out[o]; t0_out[o] (host) is the first unified time of observer o;
 * the unified step is dtau.  The library allocates and frees its own
 * scratch (one partial-sum row per block of panels).  Errors: FR_EINVAL
 * (nt < 5, even ncopies, |Minf| >= 1), FR_EWINDOW (empty window for some
 * observer, or longer than cap), FR_ENOMEM, FR_ECUDA.  Synchronises stream. */
int fwh_integrate(const double* hist, int nt, int npts, const double* y, const double* n,
                  const double* dS, double dtau, double tau0, const double* obs, int nobs,
                  const double Minf[3], double c0, double rho0, double p0, double Lspan,
                  int ncopies, double* p_out, int cap, int* nt_out, double* t0_out,
                  void* stream);

/* fwh_integrate_noalloc: the paper has no counterpart; this is a library
 * convenience.  Same arguments, results and errors as fwh_integrate, but it
 * allocates no device memory: its scratch lives in one fixed device array
 * of 2^22 doubles (32 MiB) that the library reserves on every GPU it is
 * loaded on, until the process exits.  It is for callers that cannot call
 * cudaMalloc/cudaFree, e.g. an application whose device memory is all owned
 * by its own pool allocator, or one that must not pay the device-wide
 * synchronisation of cudaFree in the middle of its work.
 *   - Limit: 8*npts*nt + ceil(npts / max(1, 32/ncopies)) * (longest
 *     observer window) must not exceed 2^22; larger problems get FR_EINVAL
 *     with a message naming the sizes (use fwh_integrate for them).
 *   - Every call looks up the array's device address in the current
 *     device's context (cudaGetSymbolAddress, which allocates nothing), so
 *     the address is never stale, e.g. after cudaDeviceReset.  Like
 *     fwh_integrate, the call reads the panel positions back to the host
 *     and synchronises the stream before it returns.
 *   - Every call on a device shares the one array: calls that overlap on
 *     the GPU (other streams or threads) race and give wrong results.  Each
 *     call writes all the scratch it reads, so nothing needs clearing.
 *   - Calls no cudaMalloc, cudaFree or other allocating routine. */
int fwh_integrate_noalloc(const double* hist, int nt, int npts, const double* y, const double* n,
                          const double* dS, double dtau, double tau0, const double* obs, int nobs,
                          const double Minf[3], double c0, double rho0, double p0, double Lspan,
                          int ncopies, double* p_out, int cap, int* nt_out, double* t0_out,
                          void* stream);

/* fwh_psd: power spectral density of observer pressure series by Welch's
 * method, as Section 3.3 computes the PSD of the pressure fluctuations (three
 * Hann windows, 50% overlap; nseg = 3 reproduces it).  Segment length
 * L = 2 floor(nt / (nseg + 1)), step L/2; periodic Hann window
 * w_n = (1 - cos(2 pi n / L)) / 2; each segment loses its mean; one-sided
 * density P_k = c_k |sum_n w_n y_n exp(-2 pi i k n / L)|^2 dt / sum_n w_n^2,
 * c_k = 2 except c_0 = c_{L/2} = 1, averaged over the segments; frequency of
 * entry k is k / (L dt), k = 0..L/2.  FP64 throughout.
 *   p          device, [nobs][ld] doubles; series o is p[o*ld .. o*ld+nt-1]
 *              (e.g. the p_out of fwh_integrate with ld = its cap)
 *   psd        device, [nobs][cap] doubles, written for k = 0..L/2
 *   nfreq_out  host int: L/2 + 1
 * Errors: FR_EINVAL for null pointers, nobs < 1, nseg < 1, ld < nt, dt <= 0,
 * L < 2 (record too short) or cap < L/2 + 1; FR_ENOMEM if its scratch
 * (twiddle table, windowed segments: 16 L + 8 nobs nseg L bytes) cannot be
 * allocated.  Synchronises the stream before returning. */
int fwh_psd(const double* p, int nobs, int nt, int ld, double dt, int nseg, double* psd, int cap,
            int* nfreq_out, void* stream);

/* Elements per thread block used by the residual kernels (0 = built-in
 * default; 1..32, or 1..15 in 3D at p = 4, where two warps share each
 * element); fr_autotune times the candidates on the current state and keeps
 * the fastest per kernel, returning it in *best. */
int fr_set_tile(fr_ctx* ctx, int elems_per_block);
int fr_autotune(fr_ctx* ctx, int* best);

/* Measurement aid (no counterpart in the paper): FP64 fused multiply-add
 * throughput of this GPU in GFLOP/s (2 flops per FMA), from a kernel of
 * independent FMA chains timed with CUDA events on stream.  The FP64 FR path
 * is bound by this rate rather than by memory bandwidth. */
int fr_probe_fp64_peak(double* gflops, void* stream);

/* Counts of kernels launched by this context since creation (for
 * benchmarking claims). */
int64_t fr_launch_count(const fr_ctx* ctx);

/* Measurement aid: captures one RK4 step as a CUDA graph with an event
 * record node around every kernel (the launch sequence of fr_rk_step_graph),
 * replays it nsteps times on stream (synchronising after each replay to read
 * the events) and returns the summed device time (ms) per kernel kind in
 * ms_out[0..5] = traces, viscous faces, residual+RK, forces/sampling, energy
 * source, reduced-degree elements, and their launch counts in n_out[0..5].
 * Advances the state exactly like fr_rk_step. */
int fr_profile_step(fr_ctx* ctx, int nsteps, void* stream, double ms_out[6], int64_t n_out[6]);

#ifdef __cplusplus
}
#endif

#endif /* LIBFR_FR_H */
