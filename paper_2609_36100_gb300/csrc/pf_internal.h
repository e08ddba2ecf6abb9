// Internal declarations shared by the kernel and host translation units of
// the phase-field library (not part of the public C ABI).
#pragma once
#include <cuda_runtime.h>
#include <cstddef>

namespace pf {

constexpr int kMaxStages = 8;
constexpr int kMaxRadices = 10;

// One FFT axis: length n = product of radices (each in {2,3,4,5,8}) and the
// device table tw[k] = exp(-2 pi i k / n), k = 0..n-1, in both precisions.
struct AxisPlan {
    int n;
    int nst;
    int rad[kMaxRadices];
    int has16;                   // some stage is radix-16 (kernels compiled with radix-16 support)
    unsigned mulm[kMaxRadices];  // division magic for n / rad[s]
    unsigned mulN[kMaxRadices];  // division magic for the stage's Ns
    const double2* tw64;
    const float2* tw32;
};

// ceil(2^32 / d) for d >= 2 (0 for d = 1, which FastDiv special-cases)
inline unsigned magic_u32(unsigned d) { return d <= 1 ? 0u : (unsigned)((0xffffffffull + d) / d); }
// radix schedule (8s first, then 4/2, 3s, 5s) and division magic of one axis
bool make_axis_plan(int n, AxisPlan& p, bool prefer16 = false);
bool make_axis_plan_radices(int n, const int* rad, int nr, AxisPlan& p);
// length of compiled (compile-time) plan `pid` (0 if unknown), and how many there are
int compiled_plan_len(int pid);
int compiled_plan_count();

// Grid geometry and the per-axis wave-number tables k_m = 2 pi m / (n d)
// (FP64, Nyquist index taken as +pi/d).
struct Geo {
    int nx, ny, nz, nxh;
    long long NK;  // nz * ny * nxh  (complex entries per field)
    long long N;   // nz * ny * nx   (real entries per field)
    double invN;   // 1/N, and its FP32 rounding (no per-thread FP64 divide)
    float invN32;
    const double* kx;  // [nxh]
    const double* ky;  // [ny]
    const double* kz;  // [nz]
    const double* lam;  // [4][NK] lambda(k) per field (FP64), or null (computed on the fly)
    const float2* lamdf;  // [4][NK] lambda(k) as double-float {h, l} (FP32-bulk contexts); with lam2 only
                          // [2][NK]: X, then the one lambda the three phi fields share
    int lam2;             // 1: the phi fields share lambda (equal kappa_v), so the double-float lambda and q
                          // tables hold two rows (X, phi) and the streams read each row once per k
    const float* kx32;  // FP32 copies of the wave-number tables (FP32-bulk kernels)
    const float* ky32;
    const float* kz32;
    AxisPlan px, py, pz;
    unsigned mul_nx, mul_nxh;  // division magic for nx and nx/2+1
    const int* active;         // batch member flag: kernels return at once when *active == 0
    const int* ypar;           // batch member: when *ypar != 0 the state lives in yother (the context's
    double2* yother;           // y_new buffer) and y_new goes to the context's y buffer
    int tx_y, tx_z, tx_el;  // tuned tile widths (kx columns) of the strided passes, 0 = heuristic
    int rp;                  // tuned row pairs per CTA in the x passes, 0 = heuristic
    int tx_zf;               // tuned tile width of the forward z pass, 0 = heuristic
    int el_pid;              // compiled plan of the fused elastic pass (length nz), 0 = the z-axis plan,
                             // -1 = no fused stage (the one-kernel pass with the z-axis column transforms)
    int xf_off;              // 1: the FP32 x passes use the staged kernel instead of the fused one
    int xf_inpl;             // 1: the FP32 fused x passes run every stage in one shared buffer (in place)
    int xf_stg;              // 1: the FP32 fused right-hand-side x pass stages the stored real fields in shared memory
    int el_unfused;          // form of the compiled-plan elastic pass: 0 fuses the last forward / first inverse
                             // stage, 1 runs every stage (and the contraction) over the three fields in place,
                             // 2 runs a cluster of three CTAs, one field each (FP32 contexts)
    const float* btab;       // FP32 elastic kernel B(k) / N over kx >= 0, |ky| <= ny/2, |kz| <= nz/2 (six
                             // symmetric entries, [6][nz/2+1][ny/2+1][nx/2+1]), or null: computed per k
};

// Model constants of the real-space and elastic terms in one compute type,
// rounded once on the host: a kernel reads them from its parameter space and
// never converts or divides in FP64 per thread (the FP64 pipe of this GPU is
// narrow enough for a few dozen conversions per thread to show up).
template <typename T>
struct PhysT {
    T Bv, Bm, inv2Av, inv2Am, A0m, A0v, Am, Av;
    T wb2;    // 2 omega_bar
    T wb;     // omega_bar
    int obst; // 1: the literal obstacle barrier omega_bar S (1 - S)
    T ie;     // 1 / pair_eps
    T twoAm;  // 2 A^m
    T w[3][3];
    T C44, Cm, Ca;
    T sig[3][6];
    T cvq[3][3];
    T mN, lN;  // -M / N, -L / N (explicit-term scalings after a forward transform)
};

// Derived model constants (Sec. 4.1 with the readings of the library).
struct Phys {
    double M;             // mobility at T
    double Am, Av, A0m, A0v, Bm, Bv;
    double inv2Am, inv2Av;  // 1/(2 A^p)
    double L, wbar;
    int obst;             // 1: the literal obstacle barrier (projection after each step)
    double w[3][3];       // pairwise barrier omega_vq (zero diagonal)
    double pair_eps;      // Huber width of |phi_v phi_q|
    double kap[3][6];     // gradient tensors (Voigt)
    int kap_iso;          // every kappa_v is a multiple of the identity
    double lamc[4];       // lambda = lamc[f] k^2 when kap_iso (lamc[0] always)
    int elastic;          // 0: all eigenstrains zero
    double Caniso, Cmix, C44;  // C11 - C12 - 2 C44, C12 + C44, C44
    double sig[3][6];     // sigma*_v = C : eps*_v (Voigt)
    double cvq[3][3];     // eps*_v : C : eps*_q
    PhysT<double> t64;    // the constants above in each compute type
    PhysT<float> t32;
};

// Device-resident coefficients of one stage (or step completion) pass, written
// each round by the batch prep kernel from the member's own step size.
struct StageCoefDev {
    double cI[kMaxStages], cE[kMaxStages];
    double gamma, qgamma;
    float cEh[kMaxStages], cEl[kMaxStages];
    float cIh[kMaxStages], cIl[kMaxStages];
    float gh, gl, qgh, qgl;
};

// Coefficients of one stage assembly / step completion pass.
struct StageTerms {
    int n;                             // number of previous-stage terms
    unsigned mI, mE;                   // bit j set: cI[j] / cE[j] nonzero (integer tests keep
                                       // the per-element branches off the FP64 pipe)
    int has_gamma;                     // gamma != 0
    const double2* z[kMaxStages];      // stage vectors z_j: FP64, or in the FP32-bulk form
                                       // double-float float4 {Re h, Im h, Re l, Im l}
    const void* f[kMaxStages];         // f^E_j (compute type)
    double cI[kMaxStages];             // dt * A^I_ij (or dt * b^I_j)
    double cE[kMaxStages];             // dt * A^E_ij (or dt * b^E_j)
    float cEh[kMaxStages], cEl[kMaxStages];  // cE = cEh + cEl (double-single split, FP32-bulk terms)
    float cIh[kMaxStages], cIl[kMaxStages];  // cI = cIh + cIl
    unsigned mY;                       // bit j set: z_j is y itself (explicit first stage)
    double gamma;                      // dt * A^I_ii (0: explicit stage)
    float gh, gl, qgh, qgl;            // gamma and qgamma, double-float split
    const double* qin;                 // table of 1/(1 - gamma lambda) for this gamma, or null
    double* qout;                      // if set: write 1/(1 - qgamma lambda) (once per step);
                                       // FP32-bulk form: float2 {h, l} entries
    double qgamma;
    const StageCoefDev* dc;            // if set: cI, cE, cEh, cEl, gamma, qgamma come from here
};

// Step control of one ensemble member, on the device.
struct MemberCtl {
    double t, h, dt, e_prev, e_last;
    int after_reject, nrej, active, accepted_now, status;
    int ypar;  // which of the two state buffers holds y (flips on every accepted attempt)
    long long n_acc, n_rej, n_rhs;
};

// Butcher arrays and controller constants shared by the members of a batch.
struct BatchConst {
    int s, embedded, nrhs;
    double AE[kMaxStages][kMaxStages], AI[kMaxStages][kMaxStages];
    double bE[kMaxStages], bI[kMaxStages], btE[kMaxStages], btI[kMaxStages];
    double gdiag;
    double t_final, h_min, h_max, h0;
    double safety, k1, k2, eta_max, eta_min, eta_rej;
    int max_rejects, q;
};

// Constants of the phase-dependent stiffness (Hu-Chen iterations): cubic
// reference medium, matrix and precipitate compliances, eigenstrains
// (Voigt order xx yy zz yz xz xy, tensor shears)
struct HCConst {
    double c0[3];         // reference medium c11, c12, c44 (sigma_xy = 2 c44 eps_xy)
    double sm[3], sv[3];  // compliances s11, s12, s44 (eps_xy = s44 sigma_xy)
    double eps[3][6];
};
void hc_constants(double C11, double C12, double C44, double C11v, double C12v, double C44v,
                  const double eps[3][6], HCConst& k);
int hc_blocks();
template <typename T>
void launch_hc_tau(const Geo& g, const HCConst& k, const void* R, const double* eu, const double* ebar, double* tau,
                   cudaStream_t s);
void launch_hc_green(const Geo& g, const HCConst& k, double2* hk, cudaStream_t s);
template <typename T>
void launch_hc_stats(const Geo& g, const HCConst& k, const void* R, const double* eu, const double* eu_prev,
                     double* part, cudaStream_t s);
template <typename T>
void launch_hc_force(const Geo& g, const HCConst& k, const void* R, const double* eu, const double* ebar, void* E,
                     cudaStream_t s);
template <typename T>
void launch_hc_energy(const Geo& g, const HCConst& k, const void* R, const double* eu, const double* ebar,
                      double* part, cudaStream_t s);

enum XMode {
    XM_PHYS1 = 0,      // C2R state -> real fields, h(phi) -> R2C (or the full RHS when elasticity is off)
    XM_PHYS2 = 1,      // C2R elastic potential + stored real fields -> RHS -> R2C
    XM_WRMS = 2,       // C2R local error + weights from stored real y -> partial sums
    XM_R2C_REAL = 3,   // real FP64 fields -> R2C (set_state)
    XM_C2R_REAL = 4,   // C2R -> real FP64 fields (get_state)
    XM_ENERGY = 5,     // C2R state -> local free-energy density partial sums + h -> R2C
    XM_PHYS2R = 6      // real-space elastic potential (argument `in`, [3][N]) + stored real fields -> RHS -> R2C
};

// Host launchers (defined in pf_kernels.cu).  `T` = compute type.
template <typename T>
void launch_z_stage(const Geo& g, const Phys& ph, const double2* y, const StageTerms& st, double2* zout,
                    void* W, cudaStream_t s);
template <typename T>
void launch_y_pass(const Geo& g, void* buf, int nf, int sign, cudaStream_t s);
// returns the number of CTAs launched (the WRMS mode writes one partial sum each)
template <typename T>
int launch_x_pass(const Geo& g, const Phys& ph, int mode, const void* in, void* out, void* R, const void* Rin,
                  double* partials, double rtol, double atol, const double* real_in, double* real_out,
                  cudaStream_t s);
template <typename T>
void launch_z_elastic(const Geo& g, const Phys& ph, void* H, cudaStream_t s);
template <typename T>
bool launch_z_elastic_unfused(const Geo& g, const Phys& ph, void* H, int pid, cudaStream_t s);
// the three-CTA cluster form (one h field per CTA); false where it does not
// apply (FP64 contexts, plans of one stage, tiles over 200 KB)
template <typename T>
bool launch_z_elastic_cluster(const Geo& g, const Phys& ph, void* H, int pid, cudaStream_t s);
// forward z FFT; scale_mode 0: y = W/N to FP64 (set_state); 1: f^E scaling
// into the compute type; 2: f^E scaling into FP64 (ABI output)
template <typename T>
void launch_z_fwd(const Geo& g, const Phys& ph, const void* W, void* out, int scale_mode, cudaStream_t s,
                  int nf = 4);
// FP32-bulk step completion as a stream (new state + FP32 local error into W)
void launch_step_complete(const Geo& g, const double2* y, const StageTerms& bt, const StageTerms& dt, int want_lte,
                          double2* ynew, void* W, cudaStream_t s);
template <typename T>
void launch_z_final(const Geo& g, const Phys& ph, const double2* y, const StageTerms& bterm,
                    const StageTerms& dterm, int want_lte, double2* ynew, void* W, cudaStream_t s);
void launch_stage_pointwise(const Geo& g, const Phys& ph, const double2* y, const StageTerms& st, int fe_is_f32,
                            double2* zout, cudaStream_t s);
void launch_solve(const Geo& g, const Phys& ph, double gamma, const double2* r, double2* z, cudaStream_t s);
void launch_lambda_table(const Geo& g, const Phys& ph, double* lam, float2* lamdf, cudaStream_t s);
// FP32 table of the elastic kernel B_vq(k)/N (diagonal eigenstrains: B is
// even in each wave-number component, so |ky| and |kz| index it)
void launch_btab(const Geo& g, const Phys& ph, float* btab, cudaStream_t s);
void launch_clamp_phi(double* real, long long N, cudaStream_t s);
// FP32-bulk stage assembly as a streaming pass (double-float z_i out, FP32
// transform input W out); the inverse z transform follows as launch_z_pass
void launch_stage_assemble(const Geo& g, const double2* y, const StageTerms& st, double2* zout, void* W,
                           cudaStream_t s);
// in-place FFT along z of nf fields (sign +1 inverse)
template <typename T>
void launch_z_pass(const Geo& g, void* buf, int nf, int sign, cudaStream_t s);
// batch round: coefficients from the member's step, controller, accepted-state copy
void launch_batch_prep(const BatchConst& bc, MemberCtl* ctl, StageCoefDev* coef, cudaStream_t s);
void launch_batch_ctl(const BatchConst& bc, MemberCtl* ctl, const double* wrms_sum, double scale, cudaStream_t s);
// kernel nodes of the device-looped ensemble graph
cudaError_t add_batch_gate_node(cudaGraphNode_t* node, cudaGraph_t graph, const MemberCtl* ctl,
                                const cudaGraphConditionalHandle* hif, int n);
cudaError_t add_batch_more_node(cudaGraphNode_t* node, cudaGraph_t graph, const cudaGraphNode_t* deps, size_t ndeps,
                                const MemberCtl* ctl, int n, cudaGraphConditionalHandle hwhile,
                                unsigned long long* rounds, unsigned long long cap, int* capped);
void launch_reduce(const double* partials, int n, double scale, double* out, cudaStream_t s);
// sets *flag (cleared beforehand) if any of the n doubles is NaN or infinite
void launch_nonfinite(const double* v, long long n, int* flag, cudaStream_t s);
void launch_energy_k(const Geo& g, const Phys& ph, const double2* y, const double2* hk, double* partials,
                     cudaStream_t s);
int x_pass_blocks(const Geo& g, int f64);
// the thread's error buffer behind pf_last_error(NULL) (256 bytes)
char* create_error_buffer();
int energy_k_blocks(const Geo& g);

}  // namespace pf
