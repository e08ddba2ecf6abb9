/*
 * pf.h -- C ABI of the GB300 pseudospectral ImEx-ARK phase-field hot path.
 *
 * The model is the KKS gamma'' precipitation model of the paper (Sec. 4.1):
 * one conserved composition field X (Nb) and three non-conserved order
 * parameters phi_1..3 (the gamma'' orientation variants), free energy
 * F = int (f_b + f_el + f_ch) dV.  The state is integrated in reciprocal space
 * (Sec. 4.2) with ImEx additive Runge-Kutta methods (Sec. 4.4, Eqs. imex_ode,
 * ARK_method, ARK_embedding): the stiff linear terms of Eqs. composition and
 * order are implicit, the rest explicit, and each implicit stage solve is a
 * diagonal divide in k-space.
 *
 * Layouts (all row-major, x fastest):
 *   real fields     double [4][nz][ny][nx]            field order X, phi_1, phi_2, phi_3
 *   k-space vectors double complex [4][nz][ny][nx/2+1] (interleaved re, im)
 *                   y^(k) = (1/N) sum_r y(r) exp(-i k.r), so the DC entry is
 *                   the field mean; kx = 0..nx/2, ky/kz in FFT order.
 *
 * Errors: every int-returning call returns PF_OK (0) or a negative PF_E*
 * code; pf_last_error() describes the last failure of a context.  A failed
 * step leaves the last accepted state intact.  Non-CUDA errors leave the
 * context usable.
 *
 * Ownership: a context owns every device buffer it allocates and frees them in
 * pf_destroy.  Caller buffers are only read or written during a call.  All
 * device work of a context is ordered on the CUDA stream given to pf_create.
 */
#ifndef PF_H
#define PF_H

#ifdef __cplusplus
extern "C" {
#endif

#define PF_OK 0
#define PF_EINVAL (-1)       /* bad argument (size, pointer, parameter)            */
#define PF_ENOMEM (-2)       /* device or host allocation failed                   */
#define PF_ECUDA (-3)        /* a CUDA runtime call failed                          */
#define PF_ENONFINITE (-4)   /* NaN/Inf in the state or error estimate              */
#define PF_ESTEPFAIL (-5)    /* step size fell below h_min or too many rejections  */
#define PF_ETIMEOUT (-6)     /* a bounded device loop ran out (pf_batch_round_cap)   */
#define PF_EUNSUPPORTED (-7) /* grid size not 2,3,5-smooth/even, or method unknown */

/* time integration methods (Sec. 4.4) */
#define PF_EULER 1 /* ImEx (forward-backward) Euler, 1 RHS per step, no embedding */
#define PF_ARK2 2  /* ARK2 of Giraldo, Kelly & Constantinescu (2013), 3 RHS per step, 1st-order embedding */
#define PF_ARK3 3  /* ARK3(2)4L[2]SA of Kennedy & Carpenter, 4 RHS per step, 2nd-order embedding */
#define PF_ARK4 4  /* ARK4(3)6L[2]SA of Kennedy & Carpenter, 6 RHS per step, 3rd-order embedding */

/* arithmetic of the transforms and right-hand side */
#define PF_FP64 0     /* everything in FP64 */
#define PF_FP32BULK 1 /* FFTs and nonlinear RHS in FP32; state, stage vectors,
                         stage combinations, composition mean, WRMS norm and
                         controller in FP64 */

typedef struct pf_ctx pf_ctx;

/* Periodic grid: each n even, 2,3,5-smooth, 4 <= n <= 1024; spacing in nm. */
typedef struct {
    int nx, ny, nz;
    double dx, dy, dz;
} pf_grid;

/* Model constants (units nm, s, GPa, K) and integrator settings.
 * Tensors use Voigt order (xx, yy, zz, yz, xz, xy) with tensor (not
 * engineering) shear components. */
typedef struct {
    /* parabolic single-phase chemical free energies f^p = A0^p + A^p (X^p - B^p)^2
       (Eq. f_ch_p read as parabolic) */
    double A_m, A_v, A0_m, A0_v;
    double B_m0, B_v, dBm_dT; /* B^m(T) = B_m0 + dBm_dT (T - T0) */
    /* mobilities: M(T) = M0 exp(-Q/R (1/T - 1/T0)) (Eq. x_gov), L (Eq. phi_gov) */
    double M0, Q_act, T, T0, L;
    /* barrier terms of Eq. f_b */
    double kappa[3][6];  /* gradient-energy tensor per variant [GPa nm^2] */
    double omega_bar;    /* double-well height: omega_bar sum_v phi_v^2 (1-phi_v)^2 */
    double omega_pair[3]; /* omega_12, omega_13, omega_23 of |phi_v phi_q| */
    double pair_eps;      /* |x| of omega_vq |phi_v phi_q| is Huber-regularised with this
                             width: d/dphi_v = omega_vq clip(phi_v phi_q / pair_eps, -1, 1) phi_q */
    /* elasticity (Eq. u_gov, homogeneous cubic modulus) */
    double C11, C12, C44;
    double eps_star[3][6]; /* eigenstrain per variant */
    /* integrator */
    int method;    /* PF_EULER, PF_ARK2, PF_ARK3 or PF_ARK4 */
    int precision; /* PF_FP64 or PF_FP32BULK */
    double rtol, atol; /* WRMS weights w = 1/(rtol |y| + atol) (Eq. wrms_weights) */
    /* PI step-size controller (the paper uses ARKODE's; these constants are
       proposed): h_new = h min(eta_max, max(eta_min, safety e^{-k1/q} e_prev^{k2/q})),
       q = embedded order + 1; after a rejection h *= max(eta_reject_min,
       safety e^{-1/q}) and the next growth is capped at 1. */
    double h0, h_min, h_max;
    int max_rejects;
    double safety, k1, k2, eta_max, eta_min, eta_reject_min;
    /* phase-dependent stiffness (Eq. u_gov with C(r) the Reuss mix of the
       matrix constants C11/C12/C44 above and the precipitate constants
       below), solved by Hu-Chen fixed-point iterations in FP64 around the
       reference medium (C^m + C^v)/2 with a stress-free mean strain; stop
       when max |eps(u)_n - eps(u)_{n-1}| <= el_tol max |eps0| or after
       el_max_iter solves.  el_inhom = 0: homogeneous modulus (closed-form
       Green kernel, one solve).  el_warm = 1: each solve starts from the
       eps(u) of the context's previous solve (warm start; one iteration
       suffices when the fields moved little), which pf_set_state and
       pf_set_state_hat discard; 0: every solve starts cold from
       tau = C0:eps0. */
    int el_inhom;
    double C11_v, C12_v, C44_v;
    double el_tol;
    int el_max_iter;
    int el_warm;
    /* barrier term of Eq. f_b: 0 = the double well omega_bar sum_v
       phi_v^2 (1 - phi_v)^2 (tanh interfaces); 1 = the literal obstacle
       term omega_bar S (1 - S), S = sum_v phi_v, with the order parameters
       clamped to [0, 1] in real space after every completed step (the
       composition's coefficients untouched).  Batches refuse 1. */
    int barrier;
} pf_params;

typedef struct {
    long long steps_accepted, steps_rejected;
    long long rhs_evals;   /* explicit RHS evaluations (including rejected attempts) */
    double t, h;           /* current time and next step size */
    double last_wrms;      /* ||LTE||_WRMS of the last attempt */
    double wall_s;         /* wall time inside pf_advance / pf_batch_advance */
    long long point_stages; /* grid points x RHS evaluations */
} pf_stats;

/* Create a context on `cuda_stream` (a cudaStream_t, NULL = legacy default
 * stream).  Validates sizes and parameters, allocates all device buffers,
 * builds FFT plans and twiddle tables (FP64, computed on the host).
 * Returns PF_EUNSUPPORTED for non-smooth/odd sizes. */
int pf_create(const pf_grid* grid, const pf_params* params, void* cuda_stream, pf_ctx** out);
void pf_destroy(pf_ctx* ctx);

/* Set the state from real-space fields (layout above); `on_device` says
 * whether `fields` is a device pointer.  Forward FFT in FP64, y = FFT/N.
 * Input holding a NaN or infinity is refused with PF_ENONFINITE and the
 * previous state is kept. */
int pf_set_state(pf_ctx* ctx, const double* fields, int on_device);
/* Copy the real-space state out (inverse FFT in FP64). Caller owns `fields`. */
int pf_get_state(pf_ctx* ctx, double* fields, int on_device);
/* Copy the k-space state vector y (layout above) in or out.  As with
 * pf_set_state, non-finite input is refused with PF_ENONFINITE and the
 * previous state is kept. */
int pf_set_state_hat(pf_ctx* ctx, const void* y_hat, int on_device);
int pf_get_state_hat(pf_ctx* ctx, void* y_hat, int on_device);

/* f^E(y): the explicit (non-stiff) right-hand side of Eqs. composition and
 * order for a device k-space vector `y_hat`, written to device `fE_hat`
 * (both complex128 ABI layout; may not alias).  Computed in the context's
 * precision:
 *   fE_X  = -M k^2 FT[mu - 2 A^m X]
 *   fE_phi_v = -L FT[dfb/dphi_v + h'(phi_v)(f^v - f^m - mu (X^v - X^m)) + h'(phi_v) e_v]
 * with e_v = IFFT[sum_q B_vq(k/|k|) FT[h(phi_q)]], B(0) = 0 (Sec. 4.1). */
int pf_rhs_explicit(pf_ctx* ctx, const void* y_hat, void* fE_hat);

/* Stage linear solve (Sec. 4.4, the SUNLinearSolver role): z = r / (1 - gamma
 * lambda(k)) with lambda_X = -2 A^m M k^2, lambda_phi_v = -L k.kappa_v.k.
 * Device complex128 vectors in ABI layout; r and z may alias. FP64. */
int pf_solve_implicit(pf_ctx* ctx, double gamma, const void* r_hat, void* z_hat);

/* One fixed step of size dt from the current state (always accepted).  If the
 * method has an embedding and `lte_wrms_out` is non-NULL, the WRMS norm of
 * the local error estimate (real space, all four fields, weights from the
 * previous solution) is written there; else 0. */
int pf_step(pf_ctx* ctx, double dt, double* lte_wrms_out);

/* Adaptive integration to t_final (accept if ||LTE||_WRMS <= 1, PI
 * controller).  Methods without an embedding take fixed steps of h0.
 * `out` may be NULL. */
int pf_advance(pf_ctx* ctx, double t_final, double rtol, double atol, pf_stats* out);

/* As pf_advance, but stop after at most max_attempts step attempts
 * (accepted or rejected); the clock and controller state carry over. */
int pf_advance_attempts(pf_ctx* ctx, double t_final, double rtol, double atol, int max_attempts, pf_stats* out);

/* Advance n independent contexts (same stream, same method and precision,
 * any grid sizes) to t_final, each with its own step size and controller.
 * One round = one step attempt of every live member (stage sequence,
 * completion, WRMS norm, accept/reject, next step size -- all on the device),
 * captured once per call into a CUDA graph.  Members run as independent
 * branches of that graph, so small grids share the GPU.  The rounds run from
 * a single launch of a device-looped graph (a conditional WHILE node over the
 * rounds, a conditional IF node per member that skips finished members) and
 * the host waits once; where the driver lacks conditional nodes, or in
 * PF_BATCH_POLLED mode, the round graph is relaunched under a host poll.
 * Members with el_inhom set are refused (PF_EUNSUPPORTED).  At
 * most pf_batch_round_cap() rounds (PF_ETIMEOUT beyond).  `out` has n entries or is NULL. */
int pf_batch_advance(pf_ctx* const* ctxs, int n, double t_final, double rtol, double atol, pf_stats* out);

/* Driver of pf_batch_advance for this process: PF_BATCH_AUTO (device-looped
 * graph where available) or PF_BATCH_POLLED.  Returns the previous mode, or
 * PF_EINVAL for an unknown one.  Not thread-safe against concurrent
 * pf_batch_advance calls. */
#define PF_BATCH_AUTO 0
#define PF_BATCH_POLLED 1
int pf_batch_mode(int mode);
/* Rounds run by the last pf_batch_advance call of this process and whether
 * they ran device-looped (1) or host-polled (0); NULL pointers allowed. */
int pf_batch_last(long long* rounds, int* looped);
/* Round cap of pf_batch_advance for this process (default 2^20): a batch
 * still live after that many rounds stops with PF_ETIMEOUT, each member left
 * at its last accepted state and clock.  cap <= 0 only queries.  Returns the
 * previous cap.  Not thread-safe against concurrent pf_batch_advance calls. */
long long pf_batch_round_cap(long long cap);

/* Total free energy F = int (f_b + f_el + f_ch) dV of the current state
 * (Sec. 4.1), FP64. */
int pf_free_energy(pf_ctx* ctx, double* F_out);

/* Integrator clock (for checkpoint/resume).  pf_set_time also resets the
 * controller history (e_prev = 1, no pending rejection). */
int pf_get_time(pf_ctx* ctx, double* t, double* h);
int pf_set_time(pf_ctx* ctx, double t, double h);
/* Elastic solves of the last right-hand-side evaluation (the Hu-Chen
 * iteration count with el_inhom set, else 1), or a negative error. */
int pf_elastic_iterations(pf_ctx* ctx);
/* Controller history for an exact resume: the last accepted ||LTE||_WRMS
 * (e_prev of the PI rule) and whether the last attempt was rejected (growth
 * capped at 1 next).  A checkpoint is pf_get_state_hat + pf_get_time +
 * pf_get_controller; restoring the three (pf_set_time before
 * pf_set_controller) continues bitwise as if never interrupted. */
int pf_get_controller(pf_ctx* ctx, double* e_prev, int* after_reject);
int pf_set_controller(pf_ctx* ctx, double e_prev, int after_reject);
int pf_get_stats(pf_ctx* ctx, pf_stats* out);
/* Step attempts of the last pf_advance as (t, h, ||LTE||_WRMS, accepted)
 * quadruples; writes at most max_attempts of them to buf (NULL allowed) and
 * returns the total count.  Lets a caller replay the decision sequence. */
int pf_get_attempts(pf_ctx* ctx, double* buf, int max_attempts);

/* Kernel profiler: CUDA events around every launch of the step driver on the
 * context's stream, with the algorithmic bytes of each launch (each field read
 * or written once per pass as the method requires).  Kernel kinds: */
#define PF_K_Z_STAGE 0    /* stage assembly + implicit solve (+ inverse z FFT in FP64) */
#define PF_K_Y 1          /* y FFT (either direction)                           */
#define PF_K_X_PHYS1 2    /* C2R x + real-space physics (h or full RHS) + R2C  */
#define PF_K_X_PHYS2 3    /* C2R x of e_v + KKS/barrier RHS + R2C              */
#define PF_K_Z_ELASTIC 4  /* forward z, Green's contraction, inverse z         */
#define PF_K_Z_FWD 5      /* forward z + k-space scaling -> f^E                 */
#define PF_K_Z_FINAL 6    /* step completion + embedded error + inverse z       */
#define PF_K_X_WRMS 7     /* C2R x of the error + WRMS partial sums             */
#define PF_K_REDUCE 8     /* deterministic WRMS reduction                       */
#define PF_K_POINTWISE 9  /* stage assembly without a RHS evaluation            */
#define PF_K_Z_IFFT 10    /* inverse z FFT of an assembled stage (FP32-bulk)    */
#define PF_NKERNELS 11
/* Turn the profiler on/off (clears pending records). */
int pf_profile_enable(pf_ctx* ctx, int on);
/* Synchronise and return, per kind, the summed event time (ms), algorithmic
 * bytes and launch count since the last read (arrays of PF_NKERNELS; NULL
 * allowed); clears the records. */
int pf_profile_read(pf_ctx* ctx, double* ms, double* bytes, long long* launches);
const char* pf_kernel_name(int kind);

/* Launch schedule of a context: tuned tile widths of the z stage-assembly
 * and completion / y / elastic passes, rows per CTA of the x passes (0 =
 * built-in heuristic), the radix order of each axis (count + up to 10 radices
 * in {2,3,4,5,8,16}, for x, y, z: ints 4-36), the tile width of the forward
 * z pass (int 37), the compiled radix plan of the elastic pass (int 38;
 * 0 = the z axis's own plan, -1 = no compiled elastic plan: the z axis's
 * column transforms, one field after another), whether the FP32 x passes run the staged kernel instead of the
 * fused one (int 39), the form of the compiled-plan elastic pass (int 40:
 * 0 fuses the last forward and first inverse stage in registers, 1 runs each
 * transform stage and the contraction over the three fields in place, 2 runs
 * a cluster of three CTAs, one h field each, sharing the contraction through
 * distributed shared memory; FP32 contexts, FP64 contexts run 0 for 2;
 * other values are refused with PF_EINVAL), whether the FP32 fused x pass of the right-hand side copies its stored
 * real fields into shared memory with its input rows (int 41) and whether the
 * FP32 fused x passes run every stage in place in one shared buffer (int 42).
 * PF_TUNE_LEN ints. */
#define PF_TUNE_LEN 43
int pf_get_tuning(pf_ctx* ctx, int* cfg, int n);
int pf_set_tuning(pf_ctx* ctx, const int* cfg, int n);
/* Autotuner: times `reps` step attempts per candidate schedule on the
 * context's buffers (coordinate descent over tile widths, rows per CTA and
 * radix orders; the state is not modified) and keeps the fastest.  Times per
 * attempt before/after are returned in ms (NULL allowed). */
int pf_autotune(pf_ctx* ctx, int reps, double* ms_before, double* ms_after);

/* Host-side query of a method's Butcher arrays (row-major s x s, length-s
 * vectors; bt/dt embedding NULL-able buffers).  Returns the stage count s,
 * or PF_EUNSUPPORTED. Buffers must hold s*s (A) and s (b) doubles; s <= 8. */
int pf_method_tableau(int method, double* AE, double* AI, double* bE, double* bI, double* btE, double* btI);

/* ---------------------------------------------------------------------------
 * Fourier-neural-operator surrogate (not in the paper).  The network maps the
 * normalised 4-field real-space state to the normalised state change over a
 * horizon tau; all layers, gradients and the Adam update run in the library's
 * kernels.  Architecture:
 *   a_0 = P x + p;  per layer l < L: A = F_K(a_l) (truncated DFT: kx < m,
 *   ky, kz in {0..m-1, n-m..n-1}), O = W_l A (per-mode complex C x C),
 *   s = (1/N) Re sum_K w_kx O e^{ik.r} (w = 1 at kx = 0, else 2),
 *   z = V_l a_l + v_l + s, a_{l+1} = GELU(z) except after the last layer;
 *   h = GELU(Q1 a_L + q1), out = Q2 h + q2.   GELU(z) = z/2 (1 + erf(z/sqrt 2)).
 * Parameters: one FP32 vector, in order P[C][4], p[C], then per layer
 * W_l[K][C][C] complex (re, im interleaved; K = 4 m^3), V_l[C][C], v_l[C], then
 * Q1[H][C], q1[H], Q2[4][H], q2[4].  With bf16 != 0 the spectral weights are
 * used in BF16 (FP32 master copy, FP32 accumulation).  Loss: mean squared
 * error.  Device arrays are FP32 [4][nz][ny][nx].
 * ------------------------------------------------------------------------- */
typedef struct pf_fno pf_fno;
int pf_fno_create(int nx, int ny, int nz, int C, int modes, int H, int L, int bf16, void* cuda_stream, pf_fno** out);
void pf_fno_destroy(pf_fno* f);
long long pf_fno_num_params(const pf_fno* f);
int pf_fno_set_params(pf_fno* f, const float* theta, long long n); /* host; resets the Adam state */
int pf_fno_get_params(pf_fno* f, float* theta, long long n);       /* host */
int pf_fno_get_grads(pf_fno* f, float* g, long long n);            /* host; gradient of the last backward */
/* per-channel input mean/std and output std used by pf_surrogate_step */
int pf_fno_set_norm(pf_fno* f, const float* in_mean, const float* in_std, const float* out_std);
int pf_fno_forward(pf_fno* f, const float* x_dev, float* out_dev); /* out_dev may be NULL */
/* gradient of the MSE against target_dev for the last forward; loss to *loss_out */
int pf_fno_backward(pf_fno* f, const float* target_dev, double* loss_out);
int pf_fno_adam(pf_fno* f, float lr, float b1, float b2, float eps);
int pf_fno_train_step(pf_fno* f, const float* x_dev, const float* target_dev, float lr, double* loss_out);
/* Normalisation statistics from solver snapshots (device FP32
 * [n_traj][n_snap][4][nz][ny][nx], n_snap >= 2): per-channel mean and
 * standard deviation of the inputs s_t and standard deviation of the
 * increments s_{t+1} - s_t over all consecutive pairs (sums in FP64), set as
 * by pf_fno_set_norm. */
int pf_fno_fit_norm(pf_fno* f, const float* snaps_dev, int n_traj, int n_snap);
/* One training step (forward, MSE backward, Adam with b1 0.9, b2 0.999,
 * eps 1e-8) on the pair (s_t, s_{t+tau}) of device FP32 [4][nz][ny][nx]
 * states: the input (s_t - mean)/std and the target (s_{t+tau} - s_t)/out_std
 * are formed on the device from the normalisation set before. */
int pf_fno_train_pair(pf_fno* f, const float* s0_dev, const float* s1_dev, float lr, double* loss_out);
const char* pf_fno_last_error(const pf_fno* f);
/* One surrogate proposal judged by the integrator (the method's own step
 * control is the judge).  The network proposes y(t + tau) = y(t) +
 * out_std * net((y(t) - mean)/std) in real space; the context then
 * integrates the same interval adaptively (pf_advance to t + tau at
 * rtol/atol, first step h), and *dist = ||y^ - y_tau||_WRMS with weights
 * w = 1/(rtol |y_tau| + atol) over all four real fields.  The proposal is
 * accepted (*accepted = 1) when *dist <= 1, i.e. when it lies within the
 * integrator's own tolerance of the verified state.  Either way the
 * context ends at the verified state y_tau and time t + tau (a proposal's
 * own error is bounded only by comparing it with an integration of the same
 * interval).  Same grid for the network and the simulation. */
int pf_surrogate_step(pf_ctx* ctx, pf_fno* f, double tau, double h, double rtol, double atol, int* accepted,
                      double* dist);

/* Allocation-free inverse transform (the paper has no counterpart; this is a
 * service for callers that cannot allocate device memory -- e.g. applications
 * that reserve their whole device budget at start-up or whose host framework
 * forbids device allocation where it calls this library -- and therefore
 * cannot create a context).  Computes what pf_set_state_hat + pf_get_state
 * compute: the real-space fields [4][nz][ny][nx] (FP64, device pointer
 * `fields`) of the k-space state `y_hat` (device complex128
 * [4][nz][ny][nx/2+1], normalised as above), on `cuda_stream`, and waits for
 * it.  All intermediates live in file-scope __device__ arrays of the library:
 * 8.25 MiB of scratch plus 96 KiB of tables, held on every GPU that loads the
 * library until the process exits.  Limits: each size even, 2,3,5-smooth,
 * 4..1024, and nz*ny*(nx/2+1) <= 135168 (a 64^3 grid); larger grids return
 * PF_EINVAL.  The first call on a device resolves the arrays' device
 * addresses (once per device).  Every call copies its twiddle tables from
 * host memory and synchronises `cuda_stream` before it returns, so no call
 * can be captured into a CUDA graph.  Every call reuses the same arrays: calls that overlap on the GPU
 * (other threads or streams) race and must be serialised by the caller; no
 * part of the scratch needs clearing, each call overwrites what it reads.
 * No cudaMalloc/cudaFree or other allocating routine is called.  Errors:
 * PF_EINVAL, PF_EUNSUPPORTED, PF_ECUDA; pf_last_error(NULL) describes them. */
int pf_state_to_real_noalloc(const pf_grid* grid, const void* y_hat, double* fields, void* cuda_stream);

/* Measurement support (the paper has no counterpart): dense FMA throughput
 * of the current device in TFLOP/s (2 flops per FMA), precision PF_FP64 or
 * PF_FP32BULK (= FP32), from eight independent FMA chains per thread over
 * 8 CTAs of 256 threads per SM; best of three timed launches after a warm-up
 * on the legacy default stream (synchronises the device).  Gives the
 * denominators of the ALU rooflines of the FP64 and FP32 kernels.
 * Returns PF_OK, PF_EINVAL, PF_ENOMEM or PF_ECUDA. */
int pf_fma_peak(int precision, double* tflops);

/* Description of the last error of `ctx` (or of the last failed pf_create
 * when ctx is NULL). Never NULL. */
const char* pf_last_error(const pf_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* PF_H */
