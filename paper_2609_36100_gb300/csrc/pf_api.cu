// Host side of the phase-field library: contexts, FFT plans and twiddle
// tables, the ImEx-ARK step driver (Sec. 4.4 of the paper), the adaptive step
// controller, and the C ABI declared in include/pf.h.
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <type_traits>
#include <algorithm>
#include <vector>

#include "pf.h"
#include "pf_internal.h"

using namespace pf;

namespace {

const double kPi = 3.14159265358979323846;
const double kRgas = 8.314462618;

thread_local char g_create_err[256] = "no error";

// ---------------------------------------------------------------------------
// Butcher tables (Sec. 4.4: the first- to fourth-order members take 1, 3, 4
// and 6 right-hand-side evaluations per step).  ImEx Euler as a 2-stage pair;
// ARK2 of Giraldo, Kelly & Constantinescu (2013), three stages, ESDIRK gamma =
// 1 - 1/sqrt(2), first-order embedding; ARK3(2)4L[2]SA and ARK4(3)6L[2]SA of
// Kennedy & Carpenter (2003), four and six stages, second- and third-order
// embeddings.  Entries are the published rationals (ARK2: the published
// expressions in sqrt(2)).
// ---------------------------------------------------------------------------
struct Tableau {
    int s = 0;
    double AE[kMaxStages][kMaxStages] = {};
    double AI[kMaxStages][kMaxStages] = {};
    double bE[kMaxStages] = {}, bI[kMaxStages] = {};
    double btE[kMaxStages] = {}, btI[kMaxStages] = {};
    bool embedded = false;
    int emb_order = 0;
};

bool make_tableau(int method, Tableau& t) {
    t = Tableau();
    if (method == PF_EULER) {
        t.s = 2;
        t.AE[1][0] = 1.0;
        t.AI[1][1] = 1.0;
        t.bE[0] = 1.0;
        t.bI[1] = 1.0;
        return true;
    }
    if (method == PF_ARK2) {
        t.s = 3;
        t.embedded = true;
        t.emb_order = 1;
        const double r2 = std::sqrt(2.0), g = 1.0 - 1.0 / r2, a = (3.0 + 2.0 * r2) / 6.0;
        t.AE[1][0] = 2.0 - r2;
        t.AE[2][0] = 1.0 - a;
        t.AE[2][1] = a;
        t.AI[1][0] = g;
        t.AI[1][1] = g;
        t.AI[2][0] = 1.0 / (2.0 * r2);
        t.AI[2][1] = 1.0 / (2.0 * r2);
        t.AI[2][2] = g;
        const double bt[3] = {(4.0 - r2) / 8.0, (4.0 - r2) / 8.0, 1.0 / (2.0 * r2)};
        for (int i = 0; i < 3; ++i) {
            t.bE[i] = t.bI[i] = t.AI[2][i];
            t.btE[i] = t.btI[i] = bt[i];
        }
        return true;
    }
    if (method == PF_ARK3) {
        t.s = 4;
        t.embedded = true;
        t.emb_order = 2;
        const double g = 1767732205903.0 / 4055673282236.0;
        double (*E)[kMaxStages] = t.AE;
        E[1][0] = 1767732205903.0 / 2027836641118.0;
        E[2][0] = 5535828885825.0 / 10492691773637.0;
        E[2][1] = 788022342437.0 / 10882634858940.0;
        E[3][0] = 6485989280629.0 / 16251701735622.0;
        E[3][1] = -4246266847089.0 / 9704473918619.0;
        E[3][2] = 10755448449292.0 / 10357097424841.0;
        double (*I)[kMaxStages] = t.AI;
        I[1][0] = g;
        I[1][1] = g;
        I[2][0] = 2746238789719.0 / 10658868560708.0;
        I[2][1] = -640167445237.0 / 6845629431997.0;
        I[2][2] = g;
        I[3][0] = 1471266399579.0 / 7840856788654.0;
        I[3][1] = -4482444167858.0 / 7529755066697.0;
        I[3][2] = 11266239266428.0 / 11593286722821.0;
        I[3][3] = g;
        const double bt[4] = {2756255671327.0 / 12835298489170.0, -10771552573575.0 / 22201958757719.0,
                              9247589265047.0 / 10645013368117.0, 2193209047091.0 / 5459859503100.0};
        for (int i = 0; i < 4; ++i) {
            t.bE[i] = t.bI[i] = I[3][i];
            t.btE[i] = t.btI[i] = bt[i];
        }
        return true;
    }
    if (method == PF_ARK4) {
        t.s = 6;
        t.embedded = true;
        t.emb_order = 3;
        double (*E)[kMaxStages] = t.AE;
        E[1][0] = 1.0 / 2.0;
        E[2][0] = 13861.0 / 62500.0;
        E[2][1] = 6889.0 / 62500.0;
        E[3][0] = -116923316275.0 / 2393684061468.0;
        E[3][1] = -2731218467317.0 / 15368042101831.0;
        E[3][2] = 9408046702089.0 / 11113171139209.0;
        E[4][0] = -451086348788.0 / 2902428689909.0;
        E[4][1] = -2682348792572.0 / 7519795681897.0;
        E[4][2] = 12662868775082.0 / 11960479115383.0;
        E[4][3] = 3355817975965.0 / 11060851509271.0;
        E[5][0] = 647845179188.0 / 3216320057751.0;
        E[5][1] = 73281519250.0 / 8382639484533.0;
        E[5][2] = 552539513391.0 / 3454668386233.0;
        E[5][3] = 3354512671639.0 / 8306763924573.0;
        E[5][4] = 4040.0 / 17871.0;
        double (*I)[kMaxStages] = t.AI;
        I[1][0] = 1.0 / 4.0;
        I[1][1] = 1.0 / 4.0;
        I[2][0] = 8611.0 / 62500.0;
        I[2][1] = -1743.0 / 31250.0;
        I[2][2] = 1.0 / 4.0;
        I[3][0] = 5012029.0 / 34652500.0;
        I[3][1] = -654441.0 / 2922500.0;
        I[3][2] = 174375.0 / 388108.0;
        I[3][3] = 1.0 / 4.0;
        I[4][0] = 15267082809.0 / 155376265600.0;
        I[4][1] = -71443401.0 / 120774400.0;
        I[4][2] = 730878875.0 / 902184768.0;
        I[4][3] = 2285395.0 / 8070912.0;
        I[4][4] = 1.0 / 4.0;
        const double b[6] = {82889.0 / 524892.0, 0.0, 15625.0 / 83664.0, 69875.0 / 102672.0, -2260.0 / 8211.0,
                             1.0 / 4.0};
        const double bt[6] = {4586570599.0 / 29645900160.0, 0.0, 178811875.0 / 945068544.0,
                              814220225.0 / 1159782912.0, -3700637.0 / 11593932.0, 61727.0 / 225920.0};
        for (int i = 0; i < 6; ++i) {
            I[5][i] = b[i];
            t.bE[i] = t.bI[i] = b[i];
            t.btE[i] = t.btI[i] = bt[i];
        }
        return true;
    }
    return false;
}

// ---------------------------------------------------------------------------
// FFT plans
// ---------------------------------------------------------------------------
// exp(-2 pi i k / n): cos and sin of the angle 2 pi k/n evaluated in long
// double (no argument reduction beyond the library's), the four quarter
// points k/n in {0, 1/4, 1/2, 3/4} set exactly, then rounded to double.
void twiddle_table(int n, std::vector<double2>& tw) {
    tw.resize(n);
    for (int k = 0; k < n; ++k) {
        const long double frac = (long double)k / (long double)n;  // in [0,1)
        const long double th = 2.0L * 3.141592653589793238462643383279502884L * frac;
        long double c = cosl(th), s = sinl(th);
        // symmetric exact points
        if (4 * k % n == 0) {
            const int q = 4 * k / n;
            c = (q == 0) ? 1.0L : (q == 2 ? -1.0L : 0.0L);
            s = (q == 1) ? 1.0L : (q == 3 ? -1.0L : 0.0L);
        }
        tw[k] = make_double2((double)c, -(double)s);
    }
}

bool smooth_even(int n) {
    if (n < 4 || n > 1024 || (n & 1)) return false;
    int m = n;
    for (int p : {2, 3, 5})
        while (m % p == 0) m /= p;
    return m == 1;
}

}  // namespace

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
struct pf_ctx {
    int dev = 0;
    cudaStream_t stream = nullptr;
    pf_grid grid{};
    pf_params prm{};
    Tableau tab;
    bool fp32 = false;
    Geo g{};
    Phys ph{};
    // stage bookkeeping
    bool need_fe[kMaxStages] = {};
    bool alias_y[kMaxStages] = {};  // z_i == y_{n-1} exactly (explicit first stage)
    // device memory
    double *d_kx = nullptr, *d_ky = nullptr, *d_kz = nullptr;
    float* d_k32 = nullptr;  // kx | ky | kz in FP32
    double2* d_tw64[3] = {};
    float2* d_tw32[3] = {};
    double2* y = nullptr;
    double2* ynew = nullptr;
    double2* zhat[kMaxStages] = {};
    void* fE[kMaxStages] = {};
    void* W = nullptr;
    void* H = nullptr;
    void* R = nullptr;
    void* R1 = nullptr;
    double* lam = nullptr;   // [4][NK] lambda(k), FP64
    float2* lamdf = nullptr;  // [4][NK] lambda(k), double-float (FP32-bulk contexts)
    float* btab = nullptr;    // FP32 elastic-kernel table (FP32-bulk contexts with diagonal eigenstrains)
    double2* xsave = nullptr;  // the composition's k-space field across the obstacle projection (barrier = 1)
    double* qtab = nullptr;  // [4][NK] 1/(1 - dt gamma lambda) of the current step (ESDIRK diagonal)
    double gdiag = 0.0;      // common nonzero implicit diagonal entry, or 0
    double* partials = nullptr;
    int npartials = 0;
    // phase-dependent stiffness (Hu-Chen iterations, FP64)
    bool inhom = false;
    HCConst hck{};
    double* hc_tau = nullptr;      // eigenstress, real [8][N] (xx yy zz yz | xz xy, two padding fields)
    double* hc_eu[2] = {};         // eps(u), real [8][N]: current and previous iterate
    double2* hc_k = nullptr;       // k-space [8][NK] (tau^, then eps^(u))
    double2* hc_ks = nullptr;      // partial-transform scratch [4][NK]
    double* hc_part = nullptr;     // per-block statistics [blocks][11]
    double* hc_ebar = nullptr;     // eps_bar on the device [6]
    double* hc_host = nullptr;     // pinned: statistics [blocks][11] and eps_bar [6]
    int hc_iters = 0;              // iterations of the last solve
    int hc_cur = 0;                // which of hc_eu holds the last solve's eps(u)
    bool hc_prev = false;          // hc_eu[hc_cur] can start the next solve (warm start)
    double* d_scalar = nullptr;
    double* h_scalar = nullptr;  // pinned
    // integrator state
    double t = 0.0, h = 0.0;
    double e_prev = 1.0;
    bool after_reject = false;
    pf_stats st{};
    std::vector<double> attempts;  // (t, h, e, accepted) quadruples of the last advance
    // kernel profiler
    bool prof_on = false;
    struct Rec {
        int kind;
        cudaEvent_t e0, e1;
        double bytes;
    };
    std::vector<Rec> prof_recs;
    std::vector<cudaEvent_t> prof_pool;
    size_t prof_next = 0;
    char err[256] = "no error";
};

namespace {

int fail(pf_ctx* c, int code, const char* fmt, ...) {
    char* dst = c ? c->err : g_create_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 256, fmt, ap);
    va_end(ap);
    return code;
}

#define PF_CUDA(ctx, call)                                                                        \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return fail(ctx, PF_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

cudaEvent_t prof_event(pf_ctx* c) {
    if (c->prof_next == c->prof_pool.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        c->prof_pool.push_back(e);
    }
    return c->prof_pool[c->prof_next++];
}

int check_launch(pf_ctx* c, const char* where) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(c, PF_ECUDA, "%s: %s", where, cudaGetErrorString(e));
    return PF_OK;
}

template <typename T>
void typed_phys(const Phys& ph, double invN, PhysT<T>& o) {
    o.Bv = (T)ph.Bv;
    o.Bm = (T)ph.Bm;
    o.inv2Av = (T)ph.inv2Av;
    o.inv2Am = (T)ph.inv2Am;
    o.A0m = (T)ph.A0m;
    o.A0v = (T)ph.A0v;
    o.Am = (T)ph.Am;
    o.Av = (T)ph.Av;
    o.wb2 = (T)(2.0 * ph.wbar);
    o.wb = (T)ph.wbar;
    o.obst = ph.obst;
    o.ie = (T)(1.0 / ph.pair_eps);
    o.twoAm = (T)(2.0 * ph.Am);
    o.C44 = (T)ph.C44;
    o.Cm = (T)ph.Cmix;
    o.Ca = (T)ph.Caniso;
    for (int a = 0; a < 3; ++a) {
        for (int b = 0; b < 3; ++b) {
            o.w[a][b] = (T)ph.w[a][b];
            o.cvq[a][b] = (T)ph.cvq[a][b];
        }
        for (int b = 0; b < 6; ++b) o.sig[a][b] = (T)ph.sig[a][b];
    }
    o.mN = (T)(-ph.M * invN);
    o.lN = (T)(-ph.L * invN);
}

void derive_phys(const pf_params& p, Phys& ph) {
    ph = Phys();
    ph.M = p.M0 * std::exp(-p.Q_act / kRgas * (1.0 / p.T - 1.0 / p.T0));
    ph.Am = p.A_m;
    ph.Av = p.A_v;
    ph.A0m = p.A0_m;
    ph.A0v = p.A0_v;
    ph.Bm = p.B_m0 + p.dBm_dT * (p.T - p.T0);
    ph.Bv = p.B_v;
    ph.inv2Am = 1.0 / (2.0 * p.A_m);
    ph.inv2Av = 1.0 / (2.0 * p.A_v);
    ph.L = p.L;
    ph.wbar = p.omega_bar;
    ph.obst = p.barrier == 1 ? 1 : 0;
    ph.pair_eps = p.pair_eps;
    ph.w[0][1] = ph.w[1][0] = p.omega_pair[0];
    ph.w[0][2] = ph.w[2][0] = p.omega_pair[1];
    ph.w[1][2] = ph.w[2][1] = p.omega_pair[2];
    std::memcpy(ph.kap, p.kappa, sizeof(ph.kap));
    ph.kap_iso = 1;
    for (int v = 0; v < 3; ++v) {
        const double* K = p.kappa[v];
        if (!(K[1] == K[0] && K[2] == K[0] && K[3] == 0.0 && K[4] == 0.0 && K[5] == 0.0)) ph.kap_iso = 0;
    }
    ph.lamc[0] = -2.0 * p.A_m * ph.M;
    for (int v = 0; v < 3; ++v) ph.lamc[1 + v] = -p.L * p.kappa[v][0];
    ph.C44 = p.C44;
    ph.Cmix = p.C12 + p.C44;
    ph.Caniso = p.C11 - p.C12 - 2.0 * p.C44;
    ph.elastic = 0;
    for (int v = 0; v < 3; ++v)
        for (int i = 0; i < 6; ++i)
            if (p.eps_star[v][i] != 0.0) ph.elastic = 1;
    // sigma* = C : eps* for cubic C (Voigt, tensor shear components)
    for (int v = 0; v < 3; ++v) {
        const double* e = p.eps_star[v];
        const double tr = e[0] + e[1] + e[2];
        for (int i = 0; i < 3; ++i) ph.sig[v][i] = (p.C11 - p.C12) * e[i] + p.C12 * tr;
        for (int i = 3; i < 6; ++i) ph.sig[v][i] = 2.0 * p.C44 * e[i];
    }
    for (int v = 0; v < 3; ++v)
        for (int q = 0; q < 3; ++q) {
            const double* e = p.eps_star[v];
            const double* s = ph.sig[q];
            ph.cvq[v][q] = e[0] * s[0] + e[1] * s[1] + e[2] * s[2] + 2.0 * (e[3] * s[3] + e[4] * s[4] + e[5] * s[5]);
        }
}

void free_all(pf_ctx* c) {
    cudaFree(c->d_kx);
    cudaFree(c->d_ky);
    cudaFree(c->d_kz);
    cudaFree(c->d_k32);
    for (int i = 0; i < 3; ++i) {
        cudaFree(c->d_tw64[i]);
        cudaFree(c->d_tw32[i]);
    }
    cudaFree(c->y);
    cudaFree(c->ynew);
    for (int i = 0; i < kMaxStages; ++i) {
        cudaFree(c->zhat[i]);
        cudaFree(c->fE[i]);
    }
    cudaFree(c->W);
    cudaFree(c->H);
    cudaFree(c->R);
    cudaFree(c->R1);
    cudaFree(c->lam);
    cudaFree(c->lamdf);
    cudaFree(c->btab);
    cudaFree(c->xsave);
    cudaFree(c->qtab);
    cudaFree(c->partials);
    cudaFree(c->hc_tau);
    cudaFree(c->hc_eu[0]);
    cudaFree(c->hc_eu[1]);
    cudaFree(c->hc_k);
    cudaFree(c->hc_ks);
    cudaFree(c->hc_part);
    cudaFree(c->hc_ebar);
    if (c->hc_host) cudaFreeHost(c->hc_host);
    cudaFree(c->d_scalar);
    if (c->h_scalar) cudaFreeHost(c->h_scalar);
    for (cudaEvent_t e : c->prof_pool) cudaEventDestroy(e);
    c->prof_pool.clear();
}

template <typename P>
int dalloc(pf_ctx* c, P** p, size_t bytes) {
    cudaError_t e = cudaMalloc((void**)p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, PF_ENOMEM, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
    }
    return PF_OK;
}

double2* fp64_scratch(pf_ctx* c) { return c->zhat[c->tab.s - 1]; }

// integer flags of the nonzero coefficients (tested per element on device)
void set_masks(StageTerms& st) {
    st.mI = st.mE = 0u;
    for (int j = 0; j < st.n; ++j) {
        if (st.cI[j] != 0.0) st.mI |= 1u << j;
        if (st.cE[j] != 0.0) st.mE |= 1u << j;
    }
    st.has_gamma = st.gamma != 0.0 ? 1 : 0;
}

// c = hi + lo with hi = fl32(c): the double-single form of an FP64 stage
// coefficient that multiplies FP32 terms
void split_ds(double c, float& hi, float& lo) {
    hi = (float)c;
    lo = (float)(c - (double)hi);
}

// Enqueue one attempted ImEx-ARK step of size dt from c->y into c->ynew; the
// WRMS sum of the local error lands in c->d_scalar when want_lte.
// Per-kernel CUDA-event timing with the algorithmic bytes of each launch
// (what the method must read and write once: every field-pass counted once).
struct ProfScope {
    pf_ctx* c;
    int kind;
    double bytes;
    cudaEvent_t e0 = nullptr;
    ProfScope(pf_ctx* c_, int kind_, double bytes_) : c(c_), kind(kind_), bytes(bytes_) {
        if (c->prof_on) {
            e0 = prof_event(c);
            cudaEventRecord(e0, c->stream);
        }
    }
    ~ProfScope() {
        if (!c->prof_on) return;
        cudaEvent_t e1 = prof_event(c);
        cudaEventRecord(e1, c->stream);
        c->prof_recs.push_back({kind, e0, e1, bytes});
    }
};

// Hu-Chen solve of the phase-dependent elasticity for the real fields R
// ([4][N] of type TR: X, phi_1..3) on the context's stream: iteration 0 with
// tau = C0:eps0 (cold start) or, with el_warm and a previous solve since the
// state was last set, no iteration 0 (the previous eps(u) takes its place),
// then tau from the previous iterate until the change of eps(u) is
// <= el_tol max |eps0| or el_max_iter solves; writes the driving
// forces e_v into E ([3][N] of type TR, if not null) and the elastic energy
// sum_r sigma:eps_el/2 (without the volume element) into *energy (if not
// null).  Each transform is the FP64 four-field pipeline of set/get state.
template <typename TR>
int hc_solve(pf_ctx* c, const void* R, void* E, double* energy) {
    const Geo& g = c->g;
    const Phys& ph = c->ph;
    cudaStream_t s = c->stream;
    const HCConst& k = c->hck;
    const int nb = hc_blocks();
    const long long N = g.N, NK = g.NK;
    double* host = c->hc_host;
    double* ebar_h = host + (size_t)nb * 11;
    auto forward = [&](const double* real, double2* out) {  // 4 real fields -> normalised k-space
        launch_x_pass<double>(g, ph, XM_R2C_REAL, nullptr, c->hc_ks, nullptr, nullptr, nullptr, 0, 0, real, nullptr, s);
        launch_y_pass<double>(g, c->hc_ks, 4, -1, s);
        launch_z_fwd<double>(g, ph, c->hc_ks, out, 0, s);
    };
    auto inverse = [&](const double2* in, double* real) {  // 4 k-space fields -> real
        StageTerms none{};
        launch_z_stage<double>(g, ph, in, none, nullptr, c->hc_ks, s);
        launch_y_pass<double>(g, c->hc_ks, 4, +1, s);
        launch_x_pass<double>(g, ph, XM_C2R_REAL, c->hc_ks, nullptr, nullptr, nullptr, nullptr, 0, 0, nullptr, real, s);
    };
    auto green = [&](double* eu) {
        forward(c->hc_tau, c->hc_k);
        forward(c->hc_tau + 4 * N, c->hc_k + 4 * NK);
        launch_hc_green(g, k, c->hc_k, s);
        inverse(c->hc_k, eu);
        inverse(c->hc_k + 4 * NK, eu + 4 * N);
    };
    // statistics -> eps_bar (host) and the change / scale
    auto stats = [&](const double* eu, const double* prev, double& change, double& scale) -> int {
        launch_hc_stats<TR>(g, k, R, eu, prev, c->hc_part, s);
        PF_CUDA(c, cudaMemcpyAsync(host, c->hc_part, (size_t)nb * 11 * sizeof(double), cudaMemcpyDeviceToHost, s));
        PF_CUDA(c, cudaStreamSynchronize(s));
        double sum[11] = {};
        for (int b = 0; b < nb; ++b)
            for (int q = 0; q < 11; ++q) sum[q] = q < 9 ? sum[q] + host[b * 11 + q] : std::fmax(sum[q], host[b * 11 + q]);
        double cav[3], sav[3], r[6];
        for (int a = 0; a < 3; ++a) cav[a] = sum[a] / (double)N;
        for (int a = 0; a < 6; ++a) r[a] = sum[3 + a] / (double)N;
        // <C> is cubic: eps_bar = <C>^-1 r with the cubic compliance of <C>
        const double d = (cav[0] - cav[1]) * (cav[0] + 2.0 * cav[1]);
        sav[0] = (cav[0] + cav[1]) / d;
        sav[1] = -cav[1] / d;
        sav[2] = 1.0 / (2.0 * cav[2]);
        const double tr = r[0] + r[1] + r[2];
        for (int a = 0; a < 3; ++a) ebar_h[a] = (sav[0] - sav[1]) * r[a] + sav[1] * tr;
        for (int a = 3; a < 6; ++a) ebar_h[a] = sav[2] * r[a];
        PF_CUDA(c, cudaMemcpyAsync(c->hc_ebar, ebar_h, 6 * sizeof(double), cudaMemcpyHostToDevice, s));
        change = sum[9];
        scale = sum[10];
        return PF_OK;
    };
    int cur = c->hc_cur;
    double change = 0.0, scale = 0.0;
    int it;
    const bool warm = c->prm.el_warm && c->hc_prev;
    c->hc_prev = false;  // set again once this solve has completed
    if (warm) {
        // warm start: eps_bar for the carried eps(u) under the current C(r)
        if (int rc = stats(c->hc_eu[cur], nullptr, change, scale)) return rc;
        it = 0;
    } else {
        launch_hc_tau<TR>(g, k, R, nullptr, nullptr, c->hc_tau, s);
        green(c->hc_eu[cur]);
        if (int rc = stats(c->hc_eu[cur], nullptr, change, scale)) return rc;
        it = 1;
    }
    const double tol = c->prm.el_tol * (scale > 0.0 ? scale : 1e-300);
    while (it < c->prm.el_max_iter) {
        const int prev = cur;
        cur ^= 1;
        launch_hc_tau<TR>(g, k, R, c->hc_eu[prev], c->hc_ebar, c->hc_tau, s);
        green(c->hc_eu[cur]);
        if (int rc = stats(c->hc_eu[cur], c->hc_eu[prev], change, scale)) return rc;
        ++it;
        if (!(change > tol)) break;  // also stops on a non-finite change
    }
    c->hc_iters = it;
    c->hc_cur = cur;
    c->hc_prev = c->prm.el_warm != 0;
    if (E) launch_hc_force<TR>(g, k, R, c->hc_eu[cur], c->hc_ebar, E, s);
    if (energy) {
        launch_hc_energy<TR>(g, k, R, c->hc_eu[cur], c->hc_ebar, c->hc_part, s);
        launch_reduce(c->hc_part, nb, 1.0, c->d_scalar + 2, s);
        PF_CUDA(c, cudaMemcpyAsync(c->h_scalar + 2, c->d_scalar + 2, sizeof(double), cudaMemcpyDeviceToHost, s));
        PF_CUDA(c, cudaStreamSynchronize(s));
        *energy = c->h_scalar[2];
    }
    return check_launch(c, "Hu-Chen elastic solve");
}

template <typename T>
int enqueue_step(pf_ctx* c, double dt, bool want_lte, const StageCoefDev* dcoef = nullptr) {
    using T2 = typename std::conditional<sizeof(T) == 8, double2, float2>::type;
    const Geo& g = c->g;
    const Phys& ph = c->ph;
    const Tableau& tb = c->tab;
    cudaStream_t s = c->stream;
    const double NK = (double)g.NK, N = (double)g.N, cb = sizeof(T2), rb = sizeof(T);
    double2* zp[kMaxStages];
    for (int i = 0; i < tb.s; ++i) zp[i] = c->alias_y[i] ? c->y : c->zhat[i];
    for (int i = 0; i < tb.s; ++i) {
        StageTerms st{};
        st.n = i;
        double terms = 0;  // bytes per k entry read from earlier stages
        for (int j = 0; j < i; ++j) {
            st.z[j] = zp[j];
            st.f[j] = c->fE[j];
            st.cI[j] = dt * tb.AI[i][j];
            st.cE[j] = dt * tb.AE[i][j];
            terms += (st.cI[j] != 0.0 && !c->alias_y[j] ? 16.0 : 0.0) + (st.cE[j] != 0.0 ? (c->fp32 ? 8.0 : 16.0) : 0.0);
        }
        st.gamma = dt * tb.AI[i][i];
        for (int j = 0; j < i; ++j) {
            split_ds(st.cE[j], st.cEh[j], st.cEl[j]);
            split_ds(st.cI[j], st.cIh[j], st.cIl[j]);
            if (c->alias_y[j]) st.mY |= 1u << j;
        }
        split_ds(st.gamma, st.gh, st.gl);
        set_masks(st);
        st.dc = dcoef ? dcoef + i : nullptr;
        if (c->gdiag != 0.0) {
            if (i == 0) {
                st.qout = c->qtab;
                st.qgamma = dt * c->gdiag;
                split_ds(st.qgamma, st.qgh, st.qgl);
            } else if (st.gamma != 0.0) {
                st.qin = c->qtab;
            }
        }
        double2* zout = c->alias_y[i] ? nullptr : zp[i];
        if (!c->need_fe[i]) {
            if (zout) {
                ProfScope p(c, PF_K_POINTWISE, 4 * NK * (16.0 + terms + 16.0));
                launch_stage_pointwise(g, ph, c->y, st, c->fp32 ? 1 : 0, zout, s);
            }
            continue;
        }
        void* Ri = (i == 0) ? c->R1 : c->R;
        if constexpr (sizeof(T) == 4) {
            // FP32-bulk: streaming double-float assembly, then the inverse z
            // transform as a plain in-place pass
            {
                ProfScope p(c, PF_K_Z_STAGE, 4 * NK * (16.0 + terms + (zout ? 16.0 : 0.0) + cb));
                launch_stage_assemble(g, c->y, st, zout, c->W, s);
            }
            {
                ProfScope p(c, PF_K_Z_IFFT, 4 * NK * 2 * cb);
                launch_z_pass<T>(g, c->W, 4, +1, s);
            }
        } else {
            ProfScope p(c, PF_K_Z_STAGE, 4 * NK * (16.0 + terms + (zout ? 16.0 : 0.0) + cb));
            launch_z_stage<T>(g, ph, c->y, st, zout, c->W, s);
        }
        {
            ProfScope p(c, PF_K_Y, 4 * NK * 2 * cb);
            launch_y_pass<T>(g, c->W, 4, +1, s);
        }
        if (c->inhom) {
            // phase-dependent stiffness: the real fields of the stage, then
            // the Hu-Chen solve (driving forces into H as real fields), then
            // the right-hand side from them
            {
                ProfScope p(c, PF_K_X_PHYS1, 4 * NK * cb + 4 * N * rb + 3 * NK * cb);
                launch_x_pass<T>(g, ph, XM_PHYS1, c->W, c->H, Ri, nullptr, nullptr, 0, 0, nullptr, nullptr, s);
            }
            {
                ProfScope p(c, PF_K_Z_ELASTIC, 0.0);
                if (int rc = hc_solve<T>(c, Ri, c->H, nullptr)) return rc;
            }
            {
                ProfScope p(c, PF_K_X_PHYS2, 3 * N * rb + 4 * N * rb + 4 * NK * cb);
                launch_x_pass<T>(g, ph, XM_PHYS2R, c->H, c->W, nullptr, Ri, nullptr, 0, 0, nullptr, nullptr, s);
            }
        } else if (ph.elastic) {
            {
                ProfScope p(c, PF_K_X_PHYS1, 4 * NK * cb + 4 * N * rb + 3 * NK * cb);
                launch_x_pass<T>(g, ph, XM_PHYS1, c->W, c->H, Ri, nullptr, nullptr, 0, 0, nullptr, nullptr, s);
            }
            {
                ProfScope p(c, PF_K_Y, 3 * NK * 2 * cb);
                launch_y_pass<T>(g, c->H, 3, -1, s);
            }
            {
                ProfScope p(c, PF_K_Z_ELASTIC, 3 * NK * 2 * cb);
                launch_z_elastic<T>(g, ph, c->H, s);
            }
            {
                ProfScope p(c, PF_K_Y, 3 * NK * 2 * cb);
                launch_y_pass<T>(g, c->H, 3, +1, s);
            }
            {
                ProfScope p(c, PF_K_X_PHYS2, 3 * NK * cb + 4 * N * rb + 4 * NK * cb);
                launch_x_pass<T>(g, ph, XM_PHYS2, c->H, c->W, nullptr, Ri, nullptr, 0, 0, nullptr, nullptr, s);
            }
        } else {
            ProfScope p(c, PF_K_X_PHYS1, 8 * NK * cb + (i == 0 ? 4 * N * rb : 0.0));
            launch_x_pass<T>(g, ph, XM_PHYS1, c->W, c->W, (i == 0) ? Ri : nullptr, nullptr, nullptr, 0, 0, nullptr,
                             nullptr, s);
        }
        {
            ProfScope p(c, PF_K_Y, 4 * NK * 2 * cb);
            launch_y_pass<T>(g, c->W, 4, -1, s);
        }
        {
            ProfScope p(c, PF_K_Z_FWD, 4 * NK * 2 * cb);
            launch_z_fwd<T>(g, ph, c->W, c->fE[i], 1, s);
        }
    }
    StageTerms bt{}, dtm{};
    bt.n = dtm.n = tb.s;
    double fterms = 0;
    const bool lte = want_lte && tb.embedded;
    for (int j = 0; j < tb.s; ++j) {
        bt.z[j] = dtm.z[j] = zp[j];
        bt.f[j] = dtm.f[j] = c->fE[j];
        bt.cI[j] = dt * tb.bI[j];
        bt.cE[j] = dt * tb.bE[j];
        if (tb.embedded) {
            dtm.cI[j] = dt * (tb.bI[j] - tb.btI[j]);
            dtm.cE[j] = dt * (tb.bE[j] - tb.btE[j]);
        }
        split_ds(bt.cE[j], bt.cEh[j], bt.cEl[j]);
        split_ds(dtm.cE[j], dtm.cEh[j], dtm.cEl[j]);
        split_ds(bt.cI[j], bt.cIh[j], bt.cIl[j]);
        split_ds(dtm.cI[j], dtm.cIh[j], dtm.cIl[j]);
        if (c->alias_y[j]) bt.mY = dtm.mY = bt.mY | (1u << j);
        set_masks(bt);
        set_masks(dtm);
        bt.dc = dcoef ? dcoef + tb.s : nullptr;
        dtm.dc = dcoef ? dcoef + tb.s + 1 : nullptr;
        const bool zI = bt.cI[j] != 0.0 || (lte && dtm.cI[j] != 0.0);
        const bool fEn = bt.cE[j] != 0.0 || (lte && dtm.cE[j] != 0.0);
        fterms += (zI && !(c->alias_y[j]) ? 16.0 : 0.0) + (fEn ? (c->fp32 ? 8.0 : 16.0) : 0.0);
    }
    if constexpr (sizeof(T) == 4) {
        // FP32-bulk: streaming completion, then the error's inverse z
        // transform as a plain in-place pass
        {
            ProfScope p(c, PF_K_Z_FINAL, 4 * NK * (16.0 + fterms + 16.0 + (lte ? cb : 0.0)));
            launch_step_complete(g, c->y, bt, dtm, lte ? 1 : 0, c->ynew, c->W, s);
        }
        if (lte) {
            ProfScope p(c, PF_K_Z_IFFT, 4 * NK * 2 * cb);
            launch_z_pass<T>(g, c->W, 4, +1, s);
        }
    } else {
        ProfScope p(c, PF_K_Z_FINAL, 4 * NK * (16.0 + fterms + 16.0 + (lte ? cb : 0.0)));
        launch_z_final<T>(g, ph, c->y, bt, dtm, lte ? 1 : 0, c->ynew, c->W, s);
    }
    if (lte) {
        {
            ProfScope p(c, PF_K_Y, 4 * NK * 2 * cb);
            launch_y_pass<T>(g, c->W, 4, +1, s);
        }
        int nb = 0;
        {
            ProfScope p(c, PF_K_X_WRMS, 4 * NK * cb + 4 * N * rb);
            nb = launch_x_pass<T>(g, ph, XM_WRMS, c->W, nullptr, nullptr, c->R1, c->partials, c->prm.rtol,
                                  c->prm.atol, nullptr, nullptr, s);
        }
        {
            ProfScope p(c, PF_K_REDUCE, nb * 8.0);
            launch_reduce(c->partials, nb, 1.0 / (4.0 * (double)g.N), c->d_scalar, s);
        }
    }
    return check_launch(c, "step kernels");
}

int step_once(pf_ctx* c, double dt, bool want_lte, double* e_out) {
    int rc = c->fp32 ? enqueue_step<float>(c, dt, want_lte) : enqueue_step<double>(c, dt, want_lte);
    if (rc) return rc;
    int nrhs = 0;
    for (int i = 0; i < c->tab.s; ++i) nrhs += c->need_fe[i] ? 1 : 0;
    c->st.rhs_evals += nrhs;
    c->st.point_stages += (long long)nrhs * c->g.N;
    double e = 0.0;
    if (want_lte && c->tab.embedded) {
        PF_CUDA(c, cudaMemcpyAsync(c->h_scalar, c->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        PF_CUDA(c, cudaStreamSynchronize(c->stream));
        e = std::sqrt(c->h_scalar[0]);
    }
    if (e_out) *e_out = e;
    return PF_OK;
}

// controller (mirrors the documented PI rule)
double ctl_accept(pf_ctx* c, double h, double e) {
    const pf_params& p = c->prm;
    const double q = c->tab.emb_order + 1;
    e = e < 1e-10 ? 1e-10 : e;
    double eta = p.safety * std::pow(e, -p.k1 / q) * std::pow(c->e_prev, p.k2 / q);
    const double cap = c->after_reject ? 1.0 : p.eta_max;
    eta = std::fmin(cap, std::fmax(p.eta_min, eta));
    c->e_prev = e;
    c->after_reject = false;
    return h * eta;
}

double ctl_reject(pf_ctx* c, double h, double e) {
    const pf_params& p = c->prm;
    c->after_reject = true;
    if (!std::isfinite(e)) return h * 0.25;
    const double q = c->tab.emb_order + 1;
    return h * std::fmax(p.eta_reject_min, p.safety * std::pow(e, -1.0 / q));
}

}  // namespace

namespace {
template <typename T>
int rhs_explicit_t(pf_ctx* c, const double2* yh, double2* out) {
    const Geo& g = c->g;
    const Phys& ph = c->ph;
    cudaStream_t s = c->stream;
    StageTerms none{};
    if constexpr (sizeof(T) == 4) {
        launch_stage_assemble(g, yh, none, nullptr, c->W, s);
        launch_z_pass<T>(g, c->W, 4, +1, s);
    } else {
        launch_z_stage<T>(g, ph, yh, none, nullptr, c->W, s);
    }
    launch_y_pass<T>(g, c->W, 4, +1, s);
    if (c->inhom) {
        launch_x_pass<T>(g, ph, XM_PHYS1, c->W, c->H, c->R, nullptr, nullptr, 0, 0, nullptr, nullptr, s);
        if (int rc = hc_solve<T>(c, c->R, c->H, nullptr)) return rc;
        launch_x_pass<T>(g, ph, XM_PHYS2R, c->H, c->W, nullptr, c->R, nullptr, 0, 0, nullptr, nullptr, s);
    } else if (ph.elastic) {
        launch_x_pass<T>(g, ph, XM_PHYS1, c->W, c->H, c->R, nullptr, nullptr, 0, 0, nullptr, nullptr, s);
        launch_y_pass<T>(g, c->H, 3, -1, s);
        launch_z_elastic<T>(g, ph, c->H, s);
        launch_y_pass<T>(g, c->H, 3, +1, s);
        launch_x_pass<T>(g, ph, XM_PHYS2, c->H, c->W, nullptr, c->R, nullptr, 0, 0, nullptr, nullptr, s);
    } else {
        launch_x_pass<T>(g, ph, XM_PHYS1, c->W, c->W, nullptr, nullptr, nullptr, 0, 0, nullptr, nullptr, s);
    }
    launch_y_pass<T>(g, c->W, 4, -1, s);
    launch_z_fwd<T>(g, ph, c->W, out, 2, s);
    return check_launch(c, "pf_rhs_explicit");
}
}  // namespace

char* pf::create_error_buffer() { return g_create_err; }

// grid of a context (used by the surrogate)
int pf_ctx_grid(pf_ctx* c, pf_grid* g) {
    if (!c || !g) return PF_EINVAL;
    *g = c->grid;
    return PF_OK;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* pf_last_error(const pf_ctx* ctx) { return ctx ? ctx->err : g_create_err; }

int pf_method_tableau(int method, double* AE, double* AI, double* bE, double* bI, double* btE, double* btI) {
    Tableau t;
    if (!make_tableau(method, t)) return PF_EUNSUPPORTED;
    for (int i = 0; i < t.s; ++i) {
        for (int j = 0; j < t.s; ++j) {
            if (AE) AE[i * t.s + j] = t.AE[i][j];
            if (AI) AI[i * t.s + j] = t.AI[i][j];
        }
        if (bE) bE[i] = t.bE[i];
        if (bI) bI[i] = t.bI[i];
        if (btE) btE[i] = t.embedded ? t.btE[i] : 0.0;
        if (btI) btI[i] = t.embedded ? t.btI[i] : 0.0;
    }
    return t.s;
}

int pf_create(const pf_grid* grid, const pf_params* params, void* cuda_stream, pf_ctx** out) {
    if (!grid || !params || !out) return fail(nullptr, PF_EINVAL, "pf_create: NULL argument");
    *out = nullptr;
    if (!smooth_even(grid->nx) || !smooth_even(grid->ny) || !smooth_even(grid->nz))
        return fail(nullptr, PF_EUNSUPPORTED, "grid %dx%dx%d: each size must be even, 2,3,5-smooth, 4..1024",
                    grid->nx, grid->ny, grid->nz);
    if (!(grid->dx > 0) || !(grid->dy > 0) || !(grid->dz > 0))
        return fail(nullptr, PF_EINVAL, "grid spacing must be positive");
    if (params->precision != PF_FP64 && params->precision != PF_FP32BULK)
        return fail(nullptr, PF_EINVAL, "unknown precision %d", params->precision);
    if (!(params->A_m > 0) || !(params->A_v > 0) || !(params->T > 0) || !(params->T0 > 0) || params->L < 0 ||
        params->M0 < 0 || !(params->pair_eps > 0))
        return fail(nullptr, PF_EINVAL, "invalid model constants (A_m, A_v, T, T0, pair_eps > 0; L, M0 >= 0)");
    pf_ctx* c = new (std::nothrow) pf_ctx();
    if (!c) return fail(nullptr, PF_ENOMEM, "host allocation failed");
    if (!make_tableau(params->method, c->tab)) {
        delete c;
        return fail(nullptr, PF_EUNSUPPORTED, "unknown method %d", params->method);
    }
    cudaGetDevice(&c->dev);
    c->stream = (cudaStream_t)cuda_stream;
    c->grid = *grid;
    c->prm = *params;
    c->fp32 = params->precision == PF_FP32BULK;
    derive_phys(*params, c->ph);
    c->inhom = params->el_inhom != 0 && c->ph.elastic;
    if (c->inhom) {
        if (!(params->C11_v > params->C12_v) || !(params->C11_v + 2 * params->C12_v > 0) || !(params->C44_v > 0) ||
            !(params->el_tol >= 0) || params->el_max_iter < 1 || (params->el_warm != 0 && params->el_warm != 1) ||
            (params->barrier != 0 && params->barrier != 1)) {
            delete c;
            return fail(nullptr, PF_EINVAL, "invalid precipitate stiffness or elastic-solver settings");
        }
        hc_constants(params->C11, params->C12, params->C44, params->C11_v, params->C12_v, params->C44_v,
                     params->eps_star, c->hck);
    }
    const Tableau& tb = c->tab;
    for (int i = 0; i < tb.s; ++i) {
        bool nf = tb.bE[i] != 0.0 || (tb.embedded && tb.btE[i] != 0.0);
        for (int k = i + 1; k < tb.s; ++k) nf = nf || tb.AE[k][i] != 0.0;
        c->need_fe[i] = nf;
        bool ex = tb.AI[i][i] == 0.0;
        for (int j = 0; j < i; ++j) ex = ex && tb.AI[i][j] == 0.0 && tb.AE[i][j] == 0.0;
        c->alias_y[i] = ex;
    }
    // one shared implicit diagonal (SDIRK/ESDIRK): 1/(1 - dt gamma lambda) is
    // formed once per step by the first stage and reused by every implicit stage
    c->gdiag = 0.0;
    for (int i = 0; i < tb.s; ++i) {
        const double d = tb.AI[i][i];
        if (d == 0.0) continue;
        if (c->gdiag == 0.0) c->gdiag = d;
        else if (c->gdiag != d) c->gdiag = -1.0;
    }
    if (c->gdiag < 0.0 || !c->need_fe[0]) c->gdiag = 0.0;
    Geo& g = c->g;
    g.nx = grid->nx;
    g.ny = grid->ny;
    g.nz = grid->nz;
    g.nxh = g.nx / 2 + 1;
    g.NK = (long long)g.nz * g.ny * g.nxh;
    g.N = (long long)g.nz * g.ny * g.nx;
    g.invN = 1.0 / (double)g.N;
    g.invN32 = (float)g.invN;
    typed_phys(c->ph, g.invN, c->ph.t64);
    typed_phys(c->ph, g.invN, c->ph.t32);
    g.mul_nx = magic_u32((unsigned)g.nx);
    g.mul_nxh = magic_u32((unsigned)g.nxh);
    int rc = PF_OK;
    // wave numbers k_m = 2 pi m / (n d), Nyquist +pi/d
    auto ktab = [](int n, double d, bool half) {
        std::vector<double> k(half ? n / 2 + 1 : n);
        for (int i = 0; i < (int)k.size(); ++i) {
            int m = i;
            if (!half && i > n / 2) m = i - n;
            k[i] = 2.0 * kPi * m / (n * d);
        }
        return k;
    };
    std::vector<double> kx = ktab(g.nx, grid->dx, true), ky = ktab(g.ny, grid->dy, false),
                        kz = ktab(g.nz, grid->dz, false);
    AxisPlan* plans[3] = {&g.px, &g.py, &g.pz};
    const int ns[3] = {g.nx, g.ny, g.nz};
    for (int a = 0; a < 3; ++a) {
        if (!make_axis_plan(ns[a], *plans[a], c->fp32)) {
            delete c;
            return fail(nullptr, PF_EUNSUPPORTED, "cannot factor %d", ns[a]);
        }
    }
    const size_t nk4 = 4 * (size_t)g.NK;
    const size_t tsz = c->fp32 ? sizeof(float) : sizeof(double);
    rc = rc ? rc : dalloc(c, &c->d_kx, kx.size() * sizeof(double));
    rc = rc ? rc : dalloc(c, &c->d_ky, ky.size() * sizeof(double));
    rc = rc ? rc : dalloc(c, &c->d_kz, kz.size() * sizeof(double));
    rc = rc ? rc : dalloc(c, &c->d_k32, (kx.size() + ky.size() + kz.size()) * sizeof(float));
    for (int a = 0; a < 3 && !rc; ++a) {
        rc = rc ? rc : dalloc(c, &c->d_tw64[a], ns[a] * sizeof(double2));
        rc = rc ? rc : dalloc(c, &c->d_tw32[a], ns[a] * sizeof(float2));
    }
    rc = rc ? rc : dalloc(c, &c->y, nk4 * sizeof(double2));
    rc = rc ? rc : dalloc(c, &c->ynew, nk4 * sizeof(double2));
    for (int i = 0; i < tb.s && !rc; ++i) {
        if (!c->alias_y[i]) rc = dalloc(c, &c->zhat[i], nk4 * sizeof(double2));
        if (!rc && c->need_fe[i]) rc = dalloc(c, &c->fE[i], nk4 * 2 * tsz);
    }
    rc = rc ? rc : dalloc(c, &c->W, nk4 * 2 * tsz);
    rc = rc ? rc : dalloc(c, &c->H, 3 * (size_t)g.NK * 2 * tsz);
    rc = rc ? rc : dalloc(c, &c->R, 4 * (size_t)g.N * tsz);
    rc = rc ? rc : dalloc(c, &c->R1, 4 * (size_t)g.N * tsz);
    rc = rc ? rc : dalloc(c, &c->lam, nk4 * sizeof(double));
    if (c->fp32) rc = rc ? rc : dalloc(c, &c->lamdf, nk4 * sizeof(float2));
    // elastic-kernel table: FP32-bulk, homogeneous modulus, diagonal
    // eigenstrains (B even in each wave-number component), at most 1 GB (794 MB
    // at 640^3)
    bool diag = true;
    for (int v = 0; v < 3; ++v)
        for (int a = 3; a < 6; ++a) diag = diag && params->eps_star[v][a] == 0.0;
    const long long tabn = (long long)(g.nz / 2 + 1) * (g.ny / 2 + 1) * g.nxh;
    if (c->fp32 && c->ph.elastic && !c->inhom && diag && 6 * tabn * (long long)sizeof(float) <= (1LL << 30))
        rc = rc ? rc : dalloc(c, &c->btab, 6 * (size_t)tabn * sizeof(float));
    rc = rc ? rc : dalloc(c, &c->qtab, nk4 * sizeof(double));
    if (params->barrier == 1) rc = rc ? rc : dalloc(c, &c->xsave, (size_t)g.NK * sizeof(double2));
    // worst case over any tuned rows-per-CTA setting (one row pair per CTA)
    c->npartials = g.nz * g.ny / 2;
    if (energy_k_blocks(g) > c->npartials) c->npartials = energy_k_blocks(g);
    rc = rc ? rc : dalloc(c, &c->partials, (size_t)c->npartials * sizeof(double));
    if (c->inhom) {
        const size_t n8 = 8 * (size_t)g.N * sizeof(double);
        rc = rc ? rc : dalloc(c, &c->hc_tau, n8);
        rc = rc ? rc : dalloc(c, &c->hc_eu[0], n8);
        rc = rc ? rc : dalloc(c, &c->hc_eu[1], n8);
        rc = rc ? rc : dalloc(c, &c->hc_k, 8 * (size_t)g.NK * sizeof(double2));
        rc = rc ? rc : dalloc(c, &c->hc_ks, 4 * (size_t)g.NK * sizeof(double2));
        rc = rc ? rc : dalloc(c, &c->hc_part, (size_t)hc_blocks() * 11 * sizeof(double));
        rc = rc ? rc : dalloc(c, &c->hc_ebar, 6 * sizeof(double));
        if (!rc && cudaMallocHost((void**)&c->hc_host, ((size_t)hc_blocks() * 11 + 8) * sizeof(double)) != cudaSuccess)
            rc = fail(c, PF_ENOMEM, "pinned host allocation failed");
        // the padding fields of the second four-field group stay zero
        if (!rc && (cudaMemset(c->hc_tau, 0, n8) != cudaSuccess || cudaMemset(c->hc_eu[0], 0, n8) != cudaSuccess ||
                    cudaMemset(c->hc_eu[1], 0, n8) != cudaSuccess))
            rc = fail(c, PF_ECUDA, "cudaMemset failed");
    }
    rc = rc ? rc : dalloc(c, &c->d_scalar, 4 * sizeof(double));
    if (!rc && cudaMallocHost((void**)&c->h_scalar, 4 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        rc = fail(c, PF_ENOMEM, "cudaMallocHost failed");
    }
    if (rc) {
        std::snprintf(g_create_err, sizeof g_create_err, "%s", c->err);
        free_all(c);
        delete c;
        return rc;
    }
    cudaError_t e = cudaSuccess;
    e = e ? e : cudaMemcpy(c->d_kx, kx.data(), kx.size() * sizeof(double), cudaMemcpyHostToDevice);
    e = e ? e : cudaMemcpy(c->d_ky, ky.data(), ky.size() * sizeof(double), cudaMemcpyHostToDevice);
    e = e ? e : cudaMemcpy(c->d_kz, kz.data(), kz.size() * sizeof(double), cudaMemcpyHostToDevice);
    {
        std::vector<float> k32;
        for (double v : kx) k32.push_back((float)v);
        for (double v : ky) k32.push_back((float)v);
        for (double v : kz) k32.push_back((float)v);
        e = e ? e : cudaMemcpy(c->d_k32, k32.data(), k32.size() * sizeof(float), cudaMemcpyHostToDevice);
    }
    for (int a = 0; a < 3 && !e; ++a) {
        std::vector<double2> tw;
        twiddle_table(ns[a], tw);
        std::vector<float2> tw32(tw.size());
        for (size_t i = 0; i < tw.size(); ++i) tw32[i] = make_float2((float)tw[i].x, (float)tw[i].y);
        e = cudaMemcpy(c->d_tw64[a], tw.data(), tw.size() * sizeof(double2), cudaMemcpyHostToDevice);
        e = e ? e : cudaMemcpy(c->d_tw32[a], tw32.data(), tw32.size() * sizeof(float2), cudaMemcpyHostToDevice);
        plans[a]->tw64 = c->d_tw64[a];
        plans[a]->tw32 = c->d_tw32[a];
    }
    e = e ? e : cudaMemsetAsync(c->y, 0, nk4 * sizeof(double2), c->stream);
    if (!e) {
        g.kx = c->d_kx;
        g.ky = c->d_ky;
        g.kz = c->d_kz;
        // the phi fields share lambda when their gradient tensors are equal
        g.lam2 = 0;
        if (c->fp32) {
            bool same = true;
            for (int v = 1; v < 3; ++v)
                for (int i = 0; i < 6; ++i) same = same && params->kappa[v][i] == params->kappa[0][i];
            g.lam2 = same ? 1 : 0;
        }
        launch_lambda_table(g, c->ph, c->lam, c->lamdf, c->stream);
        if (c->btab) launch_btab(g, c->ph, c->btab, c->stream);
        e = cudaGetLastError();
        g.lam = c->lam;
        g.lamdf = c->lamdf;
        g.btab = c->btab;
    }
    e = e ? e : cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        std::snprintf(g_create_err, sizeof g_create_err, "device setup: %s", cudaGetErrorString(e));
        free_all(c);
        delete c;
        return PF_ECUDA;
    }
    g.kx = c->d_kx;
    g.ky = c->d_ky;
    g.kz = c->d_kz;
    g.kx32 = c->d_k32;
    g.ky32 = c->d_k32 + kx.size();
    g.kz32 = c->d_k32 + kx.size() + ky.size();
    c->t = 0.0;
    c->h = params->h0;
    c->st.h = c->h;
    *out = c;
    return PF_OK;
}

void pf_destroy(pf_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->dev);
    cudaStreamSynchronize(ctx->stream);
    free_all(ctx);
    delete ctx;
}

// PF_ENONFINITE if any of the n device doubles at v is NaN or infinite
static int check_finite(pf_ctx* c, const double* v, long long n, const char* where) {
    int* flag = reinterpret_cast<int*>(c->d_scalar + 3);
    int* hflag = reinterpret_cast<int*>(c->h_scalar + 3);
    PF_CUDA(c, cudaMemsetAsync(flag, 0, sizeof(int), c->stream));
    launch_nonfinite(v, n, flag, c->stream);
    PF_CUDA(c, cudaMemcpyAsync(hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    PF_CUDA(c, cudaStreamSynchronize(c->stream));
    if (*hflag) return fail(c, PF_ENONFINITE, "%s: NaN or infinite input; state unchanged", where);
    return PF_OK;
}

int pf_set_state(pf_ctx* c, const double* fields, int on_device) {
    if (!c || !fields) return fail(c, PF_EINVAL, "pf_set_state: NULL argument");
    cudaSetDevice(c->dev);
    const Geo& g = c->g;
    double* real = reinterpret_cast<double*>(fp64_scratch(c));
    const double* src = fields;
    if (!on_device) {
        PF_CUDA(c, cudaMemcpyAsync(real, fields, 4 * (size_t)g.N * sizeof(double), cudaMemcpyHostToDevice,
                                   c->stream));
        src = real;
    }
    if (int rc = check_finite(c, src, 4 * g.N, "pf_set_state")) return rc;
    launch_x_pass<double>(g, c->ph, XM_R2C_REAL, nullptr, c->ynew, nullptr, nullptr, nullptr, 0, 0, src, nullptr,
                          c->stream);
    launch_y_pass<double>(g, c->ynew, 4, -1, c->stream);
    launch_z_fwd<double>(g, c->ph, c->ynew, c->y, 0, c->stream);
    int rc = check_launch(c, "pf_set_state");
    if (rc) return rc;
    PF_CUDA(c, cudaStreamSynchronize(c->stream));
    c->hc_prev = false;  // a new trajectory: the next Hu-Chen solve starts cold
    return PF_OK;
}

int pf_get_state(pf_ctx* c, double* fields, int on_device) {
    if (!c || !fields) return fail(c, PF_EINVAL, "pf_get_state: NULL argument");
    cudaSetDevice(c->dev);
    const Geo& g = c->g;
    StageTerms none{};
    launch_z_stage<double>(g, c->ph, c->y, none, nullptr, c->ynew, c->stream);
    launch_y_pass<double>(g, c->ynew, 4, +1, c->stream);
    double* real = on_device ? fields : reinterpret_cast<double*>(fp64_scratch(c));
    launch_x_pass<double>(g, c->ph, XM_C2R_REAL, c->ynew, nullptr, nullptr, nullptr, nullptr, 0, 0, nullptr, real,
                          c->stream);
    int rc = check_launch(c, "pf_get_state");
    if (rc) return rc;
    if (!on_device)
        PF_CUDA(c, cudaMemcpyAsync(fields, real, 4 * (size_t)g.N * sizeof(double), cudaMemcpyDeviceToHost,
                                   c->stream));
    PF_CUDA(c, cudaStreamSynchronize(c->stream));
    return PF_OK;
}

int pf_set_state_hat(pf_ctx* c, const void* y_hat, int on_device) {
    if (!c || !y_hat) return fail(c, PF_EINVAL, "pf_set_state_hat: NULL argument");
    cudaSetDevice(c->dev);
    // copied into the y_new buffer and checked there, so that a rejected
    // input leaves the state untouched
    PF_CUDA(c, cudaMemcpyAsync(c->ynew, y_hat, 4 * (size_t)c->g.NK * sizeof(double2),
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    if (int rc = check_finite(c, reinterpret_cast<const double*>(c->ynew), 8 * c->g.NK, "pf_set_state_hat"))
        return rc;
    std::swap(c->y, c->ynew);
    c->hc_prev = false;  // a new trajectory: the next Hu-Chen solve starts cold
    return PF_OK;
}

int pf_get_state_hat(pf_ctx* c, void* y_hat, int on_device) {
    if (!c || !y_hat) return fail(c, PF_EINVAL, "pf_get_state_hat: NULL argument");
    cudaSetDevice(c->dev);
    PF_CUDA(c, cudaMemcpyAsync(y_hat, c->y, 4 * (size_t)c->g.NK * sizeof(double2),
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    PF_CUDA(c, cudaStreamSynchronize(c->stream));
    return PF_OK;
}


int pf_rhs_explicit(pf_ctx* c, const void* y_hat, void* fE_hat) {
    if (!c || !y_hat || !fE_hat) return fail(c, PF_EINVAL, "pf_rhs_explicit: NULL argument");
    if (y_hat == fE_hat) return fail(c, PF_EINVAL, "pf_rhs_explicit: y_hat and fE_hat may not alias");
    cudaSetDevice(c->dev);
    const double2* yh = reinterpret_cast<const double2*>(y_hat);
    double2* out = reinterpret_cast<double2*>(fE_hat);
    int rc = c->fp32 ? rhs_explicit_t<float>(c, yh, out) : rhs_explicit_t<double>(c, yh, out);
    if (rc) return rc;
    PF_CUDA(c, cudaStreamSynchronize(c->stream));
    c->st.rhs_evals += 1;
    return PF_OK;
}

int pf_solve_implicit(pf_ctx* c, double gamma, const void* r_hat, void* z_hat) {
    if (!c || !r_hat || !z_hat) return fail(c, PF_EINVAL, "pf_solve_implicit: NULL argument");
    cudaSetDevice(c->dev);
    launch_solve(c->g, c->ph, gamma, reinterpret_cast<const double2*>(r_hat), reinterpret_cast<double2*>(z_hat),
                 c->stream);
    int rc = check_launch(c, "pf_solve_implicit");
    if (rc) return rc;
    PF_CUDA(c, cudaStreamSynchronize(c->stream));
    return PF_OK;
}

// The obstacle barrier's bound after a completed step: the state to real
// space (the FP64 pipeline of pf_get_state), the order parameters clamped to
// [0, 1], back to k-space (that of pf_set_state); the composition's
// coefficients are restored unchanged, so its mean stays exact.
static int project_obstacle(pf_ctx* c) {
    if (!c->ph.obst) return PF_OK;
    const Geo& g = c->g;
    cudaStream_t s = c->stream;
    PF_CUDA(c, cudaMemcpyAsync(c->xsave, c->y, (size_t)g.NK * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    StageTerms none{};
    double* real = reinterpret_cast<double*>(fp64_scratch(c));
    launch_z_stage<double>(g, c->ph, c->y, none, nullptr, c->ynew, s);
    launch_y_pass<double>(g, c->ynew, 4, +1, s);
    launch_x_pass<double>(g, c->ph, XM_C2R_REAL, c->ynew, nullptr, nullptr, nullptr, nullptr, 0, 0, nullptr, real, s);
    launch_clamp_phi(real, g.N, s);
    launch_x_pass<double>(g, c->ph, XM_R2C_REAL, nullptr, c->ynew, nullptr, nullptr, nullptr, 0, 0, real, nullptr, s);
    launch_y_pass<double>(g, c->ynew, 4, -1, s);
    launch_z_fwd<double>(g, c->ph, c->ynew, c->y, 0, s);
    PF_CUDA(c, cudaMemcpyAsync(c->y, c->xsave, (size_t)g.NK * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    return check_launch(c, "obstacle projection");
}

int pf_step(pf_ctx* c, double dt, double* lte_wrms_out) {
    if (!c) return fail(c, PF_EINVAL, "pf_step: NULL context");
    if (!(dt > 0) || !std::isfinite(dt)) return fail(c, PF_EINVAL, "pf_step: dt must be positive");
    cudaSetDevice(c->dev);
    double e = 0.0;
    int rc = step_once(c, dt, lte_wrms_out != nullptr, &e);
    if (rc) return rc;
    if (lte_wrms_out == nullptr) PF_CUDA(c, cudaStreamSynchronize(c->stream));
    std::swap(c->y, c->ynew);
    if (int prc = project_obstacle(c)) return prc;
    c->t += dt;
    c->st.steps_accepted += 1;
    c->st.t = c->t;
    c->st.last_wrms = e;
    if (lte_wrms_out) *lte_wrms_out = e;
    return PF_OK;
}

int pf_advance(pf_ctx* c, double t_final, double rtol, double atol, pf_stats* out) {
    return pf_advance_attempts(c, t_final, rtol, atol, 0x7fffffff, out);
}

int pf_advance_attempts(pf_ctx* c, double t_final, double rtol, double atol, int max_attempts, pf_stats* out) {
    if (!c) return fail(c, PF_EINVAL, "pf_advance: NULL context");
    if (max_attempts < 1) return fail(c, PF_EINVAL, "pf_advance_attempts: max_attempts < 1");
    if (!(rtol >= 0) || !(atol > 0)) return fail(c, PF_EINVAL, "pf_advance: need rtol >= 0, atol > 0");
    cudaSetDevice(c->dev);
    c->prm.rtol = rtol;
    c->prm.atol = atol;
    const bool adaptive = c->tab.embedded;
    auto t0 = std::chrono::steady_clock::now();
    c->attempts.clear();
    int nrej = 0;
    double h = adaptive ? c->h : c->prm.h0;
    int rc = PF_OK;
    int natt = 0;
    while (c->t < t_final * (1 - 1e-14) && natt++ < max_attempts) {
        h = std::fmin(h, t_final - c->t);
        double e = 0.0;
        rc = step_once(c, h, adaptive, &e);
        if (rc) break;
        if (!adaptive) PF_CUDA(c, cudaStreamSynchronize(c->stream));
        const bool ok = std::isfinite(e) && e <= 1.0;
        c->attempts.push_back(c->t);
        c->attempts.push_back(h);
        c->attempts.push_back(e);
        c->attempts.push_back(ok ? 1.0 : 0.0);
        c->st.last_wrms = e;
        double hn;
        if (ok) {
            std::swap(c->y, c->ynew);
            if ((rc = project_obstacle(c))) break;
            c->t += h;
            nrej = 0;
            c->st.steps_accepted += 1;
            hn = adaptive ? ctl_accept(c, h, e) : c->prm.h0;
        } else {
            c->st.steps_rejected += 1;
            if (++nrej > c->prm.max_rejects) {
                rc = fail(c, std::isfinite(e) ? PF_ESTEPFAIL : PF_ENONFINITE,
                          "step failed at t=%g: %d rejections (last ||LTE|| = %g)", c->t, nrej, e);
                break;
            }
            hn = ctl_reject(c, h, e);
        }
        h = std::fmin(std::fmax(hn, c->prm.h_min), c->prm.h_max);
    }
    if (adaptive) c->h = h;
    c->st.t = c->t;
    c->st.h = c->h;
    c->st.wall_s += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (out) *out = c->st;
    return rc;
}

static int g_batch_mode = PF_BATCH_AUTO;
static long long g_batch_rounds = 0;
static int g_batch_looped = 0;
static long long g_round_cap = 1LL << 20;

long long pf_batch_round_cap(long long cap) {
    const long long prev = g_round_cap;
    if (cap > 0) g_round_cap = cap;
    return prev;
}

int pf_batch_mode(int mode) {
    if (mode != PF_BATCH_AUTO && mode != PF_BATCH_POLLED) return fail(nullptr, PF_EINVAL, "pf_batch_mode: unknown mode");
    const int prev = g_batch_mode;
    g_batch_mode = mode;
    return prev;
}

int pf_batch_last(long long* rounds, int* looped) {
    if (rounds) *rounds = g_batch_rounds;
    if (looped) *looped = g_batch_looped;
    return PF_OK;
}

int pf_batch_advance(pf_ctx* const* ctxs, int n, double t_final, double rtol, double atol, pf_stats* out) {
    if (!ctxs || n <= 0) return fail(nullptr, PF_EINVAL, "pf_batch_advance: empty batch");
    if (!(rtol >= 0) || !(atol > 0)) return fail(nullptr, PF_EINVAL, "pf_batch_advance: need rtol >= 0, atol > 0");
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]) return fail(nullptr, PF_EINVAL, "pf_batch_advance: NULL context %d", i);
        if (ctxs[i]->prm.method != ctxs[0]->prm.method || ctxs[i]->fp32 != ctxs[0]->fp32)
            return fail(ctxs[i], PF_EINVAL, "pf_batch_advance: members differ in method or precision");
        if (ctxs[i]->ph.obst)
            return fail(ctxs[i], PF_EUNSUPPORTED,
                        "pf_batch_advance: the obstacle barrier's projection after each step is not part of the "
                        "batch graph");
        if (ctxs[i]->inhom)
            return fail(ctxs[i], PF_EUNSUPPORTED,
                        "pf_batch_advance: the Hu-Chen elastic solve reads its convergence on the host per iteration "
                        "and cannot run inside the batch graph");
        if (ctxs[i]->stream != ctxs[0]->stream || ctxs[i]->dev != ctxs[0]->dev)
            return fail(ctxs[i], PF_EINVAL, "pf_batch_advance: members must share the device and stream");
    }
    pf_ctx* c0 = ctxs[0];
    cudaSetDevice(c0->dev);
    cudaStream_t s = c0->stream;
    const Tableau& tb = c0->tab;
    auto t0 = std::chrono::steady_clock::now();
    // shared constants of the round kernels
    BatchConst bc{};
    bc.s = tb.s;
    bc.embedded = tb.embedded ? 1 : 0;
    bc.nrhs = 0;
    for (int i = 0; i < tb.s; ++i) bc.nrhs += c0->need_fe[i] ? 1 : 0;
    std::memcpy(bc.AE, tb.AE, sizeof bc.AE);
    std::memcpy(bc.AI, tb.AI, sizeof bc.AI);
    std::memcpy(bc.bE, tb.bE, sizeof bc.bE);
    std::memcpy(bc.bI, tb.bI, sizeof bc.bI);
    std::memcpy(bc.btE, tb.btE, sizeof bc.btE);
    std::memcpy(bc.btI, tb.btI, sizeof bc.btI);
    bc.gdiag = c0->gdiag;
    bc.t_final = t_final;
    const pf_params& p0 = c0->prm;
    bc.h_min = p0.h_min;
    bc.h_max = p0.h_max;
    bc.h0 = p0.h0;
    bc.safety = p0.safety;
    bc.k1 = p0.k1;
    bc.k2 = p0.k2;
    bc.eta_max = p0.eta_max;
    bc.eta_min = p0.eta_min;
    bc.eta_rej = p0.eta_reject_min;
    bc.max_rejects = p0.max_rejects;
    bc.q = tb.emb_order + 1;
    // per-call device state: one MemberCtl and (s + 2) coefficient sets per member
    MemberCtl* d_ctl = nullptr;
    StageCoefDev* d_coef = nullptr;
    MemberCtl* h_ctl = nullptr;
    const int ncoef = tb.s + 2;
    int rc = dalloc(c0, &d_ctl, sizeof(MemberCtl) * n);
    rc = rc ? rc : dalloc(c0, &d_coef, sizeof(StageCoefDev) * n * ncoef);
    if (!rc && cudaMallocHost((void**)&h_ctl, sizeof(MemberCtl) * n) != cudaSuccess) {
        cudaGetLastError();
        rc = fail(c0, PF_ENOMEM, "cudaMallocHost failed");
    }
    std::vector<cudaGraph_t> graphs(n, nullptr);
    cudaGraph_t batch = nullptr;
    cudaGraphExec_t exec = nullptr;
    for (int m = 0; m < n && !rc; ++m) {
        pf_ctx* c = ctxs[m];
        MemberCtl& h = h_ctl[m];
        std::memset(&h, 0, sizeof h);
        h.t = c->t;
        h.h = tb.embedded ? c->h : c->prm.h0;
        h.e_prev = c->e_prev;
        h.after_reject = c->after_reject ? 1 : 0;
        h.active = c->t < t_final * (1 - 1e-14) ? 1 : 0;
        c->prm.rtol = rtol;
        c->prm.atol = atol;
    }
    // a private stream forked from the members' stream: graphs are captured
    // and replayed there (the legacy default stream cannot be captured)
    cudaStream_t cap = nullptr;
    cudaEvent_t fork = nullptr;
    if (!rc) {
        cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(fork, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cap, fork, 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_ctl, h_ctl, sizeof(MemberCtl) * n, cudaMemcpyHostToDevice, cap);
        if (e != cudaSuccess) rc = fail(c0, PF_ECUDA, "batch set-up: %s", cudaGetErrorString(e));
    }
    const cudaStream_t s_user = s;
    if (cap) s = cap;
    // capture one round of each member: prep, stages, completion, norm,
    // controller (an accepted attempt flips which state buffer holds y)
    for (int m = 0; m < n && !rc; ++m) {
        pf_ctx* c = ctxs[m];
        const bool prof = c->prof_on;
        c->prof_on = false;
        c->g.active = &d_ctl[m].active;
        c->g.ypar = &d_ctl[m].ypar;
        c->g.yother = c->ynew;
        c->stream = cap;
        StageCoefDev* coef = d_coef + (size_t)m * ncoef;
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) {
            launch_batch_prep(bc, d_ctl + m, coef, s);
            int r2 = c->fp32 ? enqueue_step<float>(c, 1.0, tb.embedded, coef)
                             : enqueue_step<double>(c, 1.0, tb.embedded, coef);
            launch_batch_ctl(bc, d_ctl + m, c->d_scalar, 1.0, s);
            e = cudaStreamEndCapture(s, &graphs[m]);
            if (r2) rc = r2;
        }
        c->g.active = nullptr;
        c->g.ypar = nullptr;
        c->g.yother = nullptr;
        c->stream = s_user;
        c->prof_on = prof;
        if (!rc && e != cudaSuccess) rc = fail(c0, PF_ECUDA, "batch capture: %s", cudaGetErrorString(e));
    }
    // One graph launch advances the whole ensemble: a WHILE node (some member
    // live, round cap 2^20) around one round in which a gate kernel opens each
    // member's IF node only while that member is live, so members that are
    // done launch nothing, and the host waits once.  Where conditional nodes
    // are unavailable, one plain graph holding every member's round is
    // relaunched with a host poll of the live flags after every two rounds.
    struct LoopState {
        unsigned long long rounds;
        int capped;
    };
    const unsigned long long kRoundCap = (unsigned long long)g_round_cap;
    LoopState* d_loop = nullptr;
    cudaGraphConditionalHandle* d_hif = nullptr;
    bool looped = false;
    if (!rc && g_batch_mode == PF_BATCH_AUTO) {
        cudaError_t e = cudaMalloc((void**)&d_loop, sizeof(LoopState));
        if (e == cudaSuccess) e = cudaMalloc((void**)&d_hif, sizeof(cudaGraphConditionalHandle) * n);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_loop, 0, sizeof(LoopState), s);
        std::vector<cudaGraphConditionalHandle> hif(n);
        cudaGraphConditionalHandle hw{};
        cudaGraph_t top = nullptr;
        if (e == cudaSuccess) e = cudaGraphCreate(&top, 0);
        if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hw, top, 1, cudaGraphCondAssignDefault);
        cudaGraphNodeParams wp{};
        wp.type = cudaGraphNodeTypeConditional;
        wp.conditional.handle = hw;
        wp.conditional.type = cudaGraphCondTypeWhile;
        wp.conditional.size = 1;
        cudaGraphNode_t wnode{};
        if (e == cudaSuccess) e = cudaGraphAddNode(&wnode, top, nullptr, nullptr, 0, &wp);
        cudaGraph_t body = e == cudaSuccess ? wp.conditional.phGraph_out[0] : nullptr;
        for (int m = 0; m < n && e == cudaSuccess; ++m) e = cudaGraphConditionalHandleCreate(&hif[m], body, 0, 0);
        if (e == cudaSuccess)
            e = cudaMemcpy(d_hif, hif.data(), sizeof(cudaGraphConditionalHandle) * n, cudaMemcpyHostToDevice);
        cudaGraphNode_t gate{};
        if (e == cudaSuccess) e = add_batch_gate_node(&gate, body, d_ctl, d_hif, n);
        // members large enough to fill the GPU alone run one after another;
        // smaller ones run as independent branches beside them
        const long long kFillsGpu = 1LL << 21;  // grid points (128^3)
        std::vector<cudaGraphNode_t> ifn(n);
        cudaGraphNode_t prev_large = gate;
        for (int m = 0; m < n && e == cudaSuccess; ++m) {
            cudaGraphNodeParams ip{};
            ip.type = cudaGraphNodeTypeConditional;
            ip.conditional.handle = hif[m];
            ip.conditional.type = cudaGraphCondTypeIf;
            ip.conditional.size = 1;
            const bool large = ctxs[m]->g.N >= kFillsGpu;
            e = cudaGraphAddNode(&ifn[m], body, large ? &prev_large : &gate, nullptr, 1, &ip);
            if (large) prev_large = ifn[m];
            cudaGraphNode_t child{};
            if (e == cudaSuccess) e = cudaGraphAddChildGraphNode(&child, ip.conditional.phGraph_out[0], nullptr, 0, graphs[m]);
        }
        cudaGraphNode_t more{};
        if (e == cudaSuccess)
            e = add_batch_more_node(&more, body, ifn.data(), ifn.size(), d_ctl, n, hw, &d_loop->rounds, kRoundCap,
                                    &d_loop->capped);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, top, 0);
        if (e == cudaSuccess) {
            looped = true;
            batch = top;
        } else {
            cudaGetLastError();
            if (top) cudaGraphDestroy(top);
            exec = nullptr;
        }
    }
    long long rounds = 0;
    if (!rc && looped) {
        LoopState hl{};
        cudaError_t e = cudaGraphLaunch(exec, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_ctl, d_ctl, sizeof(MemberCtl) * n, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hl, d_loop, sizeof hl, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = fail(c0, PF_ECUDA, "batch launch: %s", cudaGetErrorString(e));
        rounds = (long long)hl.rounds;
        if (!rc && hl.capped) rc = fail(c0, PF_ETIMEOUT, "pf_batch_advance: no end after %llu rounds", hl.rounds);
    } else if (!rc) {
        cudaError_t e = cudaGraphCreate(&batch, 0);
        for (int m = 0; m < n && e == cudaSuccess; ++m) {
            cudaGraphNode_t node;
            e = cudaGraphAddChildGraphNode(&node, batch, nullptr, 0, graphs[m]);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, batch, 0);
        if (e != cudaSuccess) rc = fail(c0, PF_ECUDA, "batch graph: %s", cudaGetErrorString(e));
        while (!rc) {
            e = cudaGraphLaunch(exec, s);
            if (e == cudaSuccess) e = cudaGraphLaunch(exec, s);
            rounds += 2;
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(h_ctl, d_ctl, sizeof(MemberCtl) * n, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) {
                rc = fail(c0, PF_ECUDA, "batch round: %s", cudaGetErrorString(e));
                break;
            }
            int live = 0;
            for (int m = 0; m < n; ++m) live += h_ctl[m].active;
            if (!live) break;
            if (rounds >= (long long)kRoundCap) {
                rc = fail(c0, PF_ETIMEOUT, "pf_batch_advance: no end after %lld rounds", rounds);
                break;
            }
        }
    }
    g_batch_rounds = rounds;
    g_batch_looped = looped ? 1 : 0;
    const double wall = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int m = 0; m < n && h_ctl; ++m) {
        pf_ctx* c = ctxs[m];
        const MemberCtl& h = h_ctl[m];
        if (rounds > 0) {
            if (h.ypar) std::swap(c->y, c->ynew);  // the state ended in the y_new buffer
            c->t = h.t;
            if (tb.embedded) c->h = h.h;
            c->e_prev = h.e_prev;
            c->after_reject = h.after_reject != 0;
            c->st.steps_accepted += h.n_acc;
            c->st.steps_rejected += h.n_rej;
            c->st.rhs_evals += h.n_rhs;
            c->st.point_stages += h.n_rhs * c->g.N;
            c->st.last_wrms = h.e_last;
        }
        c->st.wall_s += wall;
        c->st.t = c->t;
        c->st.h = c->h;
        if (out) out[m] = c->st;
        if (!rc && h.status) rc = fail(c, h.status, "pf_batch_advance: member %d failed at t=%g", m, h.t);
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (batch) cudaGraphDestroy(batch);
    for (cudaGraph_t g : graphs)
        if (g) cudaGraphDestroy(g);
    cudaStreamSynchronize(s);
    if (cap) cudaStreamDestroy(cap);
    if (fork) cudaEventDestroy(fork);
    cudaFree(d_ctl);
    cudaFree(d_coef);
    cudaFree(d_loop);
    cudaFree(d_hif);
    if (h_ctl) cudaFreeHost(h_ctl);
    return rc;
}

int pf_free_energy(pf_ctx* c, double* F_out) {
    if (!c || !F_out) return fail(c, PF_EINVAL, "pf_free_energy: NULL argument");
    cudaSetDevice(c->dev);
    const Geo& g = c->g;
    cudaStream_t s = c->stream;
    double2* S1 = c->ynew;
    double2* S2 = fp64_scratch(c);
    StageTerms none{};
    double Fel = 0.0;
    Phys phk = c->ph;
    if (c->inhom) {
        // elastic energy of the Hu-Chen equilibrium of the current state, in
        // real space; the closed-form k-space kernel term is left out below
        double* real = reinterpret_cast<double*>(S2);
        launch_z_stage<double>(g, c->ph, c->y, none, nullptr, S1, s);
        launch_y_pass<double>(g, S1, 4, +1, s);
        launch_x_pass<double>(g, c->ph, XM_C2R_REAL, S1, nullptr, nullptr, nullptr, nullptr, 0, 0, nullptr, real, s);
        if (int rc = hc_solve<double>(c, real, nullptr, &Fel)) return rc;
        phk.elastic = 0;
    }
    launch_z_stage<double>(g, c->ph, c->y, none, nullptr, S1, s);
    launch_y_pass<double>(g, S1, 4, +1, s);
    launch_x_pass<double>(g, c->ph, XM_ENERGY, S1, S2, nullptr, nullptr, c->partials, 0, 0, nullptr, nullptr, s);
    int rc = check_launch(c, "pf_free_energy");
    if (rc) return rc;
    launch_reduce(c->partials, x_pass_blocks(g, 1), 1.0, c->d_scalar, s);  // local densities
    launch_y_pass<double>(g, S2, 3, -1, s);
    launch_z_fwd<double>(g, c->ph, S2, S1, 0, s, 3);  // h^ (normalised) into S1
    launch_energy_k(g, phk, c->y, S1, c->partials, s);
    launch_reduce(c->partials, energy_k_blocks(g), 1.0, c->d_scalar + 1, s);
    rc = check_launch(c, "pf_free_energy");
    if (rc) return rc;
    PF_CUDA(c, cudaMemcpyAsync(c->h_scalar, c->d_scalar, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    PF_CUDA(c, cudaStreamSynchronize(s));
    const double dV = c->grid.dx * c->grid.dy * c->grid.dz;
    const double V = (double)g.N * dV;
    *F_out = c->h_scalar[0] * dV + 0.5 * V * c->h_scalar[1] + Fel * dV;
    return PF_OK;
}

int pf_get_time(pf_ctx* c, double* t, double* h) {
    if (!c) return fail(c, PF_EINVAL, "pf_get_time: NULL context");
    if (t) *t = c->t;
    if (h) *h = c->h;
    return PF_OK;
}

int pf_set_time(pf_ctx* c, double t, double h) {
    if (!c || !(h > 0)) return fail(c, PF_EINVAL, "pf_set_time: bad argument");
    c->t = t;
    c->h = h;
    c->e_prev = 1.0;
    c->after_reject = false;
    return PF_OK;
}

int pf_elastic_iterations(pf_ctx* c) {
    if (!c) return fail(c, PF_EINVAL, "pf_elastic_iterations: NULL context");
    return c->inhom ? c->hc_iters : 1;
}

int pf_get_controller(pf_ctx* c, double* e_prev, int* after_reject) {
    if (!c) return fail(c, PF_EINVAL, "pf_get_controller: NULL context");
    if (e_prev) *e_prev = c->e_prev;
    if (after_reject) *after_reject = c->after_reject ? 1 : 0;
    return PF_OK;
}

int pf_set_controller(pf_ctx* c, double e_prev, int after_reject) {
    if (!c || !(e_prev > 0) || !std::isfinite(e_prev)) return fail(c, PF_EINVAL, "pf_set_controller: bad argument");
    c->e_prev = e_prev;
    c->after_reject = after_reject != 0;
    return PF_OK;
}

int pf_get_stats(pf_ctx* c, pf_stats* out) {
    if (!c || !out) return fail(c, PF_EINVAL, "pf_get_stats: NULL argument");
    c->st.t = c->t;
    c->st.h = c->h;
    *out = c->st;
    return PF_OK;
}

// ---------------------------------------------------------------------------
// autotuner: tile widths of the strided passes, rows per CTA of the x passes,
// and the radix order of each axis, chosen by timing whole step attempts on
// the context's own buffers (coordinate descent)
// ---------------------------------------------------------------------------
static void plan_to_cfg(const AxisPlan& p, int* out) {
    out[0] = p.nst;
    for (int s = 0; s < kMaxRadices; ++s) out[1 + s] = s < p.nst ? p.rad[s] : 0;
}

int pf_get_tuning(pf_ctx* c, int* cfg, int n) {
    if (!c || !cfg || n < PF_TUNE_LEN) return fail(c, PF_EINVAL, "pf_get_tuning: need %d ints", PF_TUNE_LEN);
    cfg[0] = c->g.tx_z;
    cfg[1] = c->g.tx_y;
    cfg[2] = c->g.tx_el;
    cfg[3] = c->g.rp;
    cfg[37] = c->g.tx_zf;
    cfg[38] = c->g.el_pid;
    cfg[39] = c->g.xf_off;
    cfg[40] = c->g.el_unfused;
    cfg[41] = c->g.xf_stg;
    cfg[42] = c->g.xf_inpl;
    plan_to_cfg(c->g.px, cfg + 4);
    plan_to_cfg(c->g.py, cfg + 4 + 11);
    plan_to_cfg(c->g.pz, cfg + 4 + 22);
    return PF_OK;
}

int pf_set_tuning(pf_ctx* c, const int* cfg, int n) {
    if (!c || !cfg || n < PF_TUNE_LEN) return fail(c, PF_EINVAL, "pf_set_tuning: need %d ints", PF_TUNE_LEN);
    Geo g = c->g;
    g.tx_z = cfg[0];
    g.tx_y = cfg[1];
    g.tx_el = cfg[2];
    g.rp = cfg[3];
    g.tx_zf = cfg[37];
    if (cfg[38] < -1) return fail(c, PF_EINVAL, "pf_set_tuning: bad elastic plan %d", cfg[38]);
    if (cfg[38] > 0 && compiled_plan_len(cfg[38]) != g.nz)
        return fail(c, PF_EINVAL, "pf_set_tuning: elastic plan %d does not have length nz", cfg[38]);
    g.el_pid = cfg[38];
    g.xf_off = cfg[39] != 0;
    if (cfg[40] < 0 || cfg[40] > 2) return fail(c, PF_EINVAL, "pf_set_tuning: bad elastic form %d", cfg[40]);
    g.el_unfused = cfg[40];
    g.xf_stg = cfg[41] != 0;
    g.xf_inpl = cfg[42] != 0;
    AxisPlan* pl[3] = {&g.px, &g.py, &g.pz};
    const int ns[3] = {g.nx, g.ny, g.nz};
    for (int a = 0; a < 3; ++a) {
        const int* r = cfg + 4 + 11 * a;
        AxisPlan p = *pl[a];
        if (r[0] > 0 && !make_axis_plan_radices(ns[a], r + 1, r[0], p))
            return fail(c, PF_EINVAL, "pf_set_tuning: bad radix order for axis %d", a);
        p.tw64 = pl[a]->tw64;
        p.tw32 = pl[a]->tw32;
        *pl[a] = p;
    }
    c->g = g;
    return PF_OK;
}

namespace {

// distinct orders of the radix multisets that factor n with the fewest (and
// one more) stages, at most `cap` of them
std::vector<std::vector<int>> radix_orders(int n, size_t cap) {
    int m = n, a = 0, b = 0, cc = 0;
    while (m % 2 == 0) { m /= 2; ++a; }
    while (m % 3 == 0) { m /= 3; ++b; }
    while (m % 5 == 0) { m /= 5; ++cc; }
    std::vector<std::vector<int>> sets;
    // power-of-two parts: k16 sixteens, k8 eights, k4 fours, k2 twos with
    // 4 k16 + 3 k8 + 2 k4 + k2 = a
    int best = 1 << 30;
    std::vector<std::vector<int>> twos;
    for (int k16 = 0; 4 * k16 <= a; ++k16)
        for (int k8 = 0; 4 * k16 + 3 * k8 <= a; ++k8)
            for (int k4 = 0; 4 * k16 + 3 * k8 + 2 * k4 <= a; ++k4) {
                const int k2 = a - 4 * k16 - 3 * k8 - 2 * k4;
                if (k2 > 1) continue;
                std::vector<int> v;
                for (int i = 0; i < k16; ++i) v.push_back(16);
                for (int i = 0; i < k8; ++i) v.push_back(8);
                for (int i = 0; i < k4; ++i) v.push_back(4);
                for (int i = 0; i < k2; ++i) v.push_back(2);
                twos.push_back(v);
                if ((int)v.size() < best) best = (int)v.size();
            }
    for (auto& v : twos) {
        if ((int)v.size() > best + 1) continue;
        for (int i = 0; i < b; ++i) v.push_back(3);
        for (int i = 0; i < cc; ++i) v.push_back(5);
        sets.push_back(v);
    }
    // fewest stages first, so that the cap keeps them
    std::stable_sort(sets.begin(), sets.end(),
                     [](const std::vector<int>& x, const std::vector<int>& y) { return x.size() < y.size(); });
    std::vector<std::vector<int>> out;
    for (auto v : sets) {
        std::sort(v.begin(), v.end());
        do {
            out.push_back(v);
            if (out.size() >= cap) return out;
        } while (std::next_permutation(v.begin(), v.end()));
    }
    return out;
}

double time_attempts(pf_ctx* c, int reps) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const bool prof = c->prof_on;
    c->prof_on = false;
    // warm-up, then timed step attempts (the state itself is never changed)
    int rc = c->fp32 ? enqueue_step<float>(c, 0.5, true) : enqueue_step<double>(c, 0.5, true);
    cudaEventRecord(e0, c->stream);
    for (int r = 0; r < reps && !rc; ++r)
        rc = c->fp32 ? enqueue_step<float>(c, 0.5, true) : enqueue_step<double>(c, 0.5, true);
    cudaEventRecord(e1, c->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->prof_on = prof;
    return rc ? 1e30 : (double)ms / reps;
}

}  // namespace

int pf_autotune(pf_ctx* c, int reps, double* ms_before, double* ms_after) {
    if (!c || reps < 1) return fail(c, PF_EINVAL, "pf_autotune: bad argument");
    cudaSetDevice(c->dev);
    int cfg[PF_TUNE_LEN], best[PF_TUNE_LEN];
    pf_get_tuning(c, best, PF_TUNE_LEN);
    double tbest = time_attempts(c, reps);
    if (ms_before) *ms_before = tbest;
    auto trial = [&](const int* cand) {
        if (pf_set_tuning(c, cand, PF_TUNE_LEN) != PF_OK) return;
        const double t = time_attempts(c, reps);
        if (t < tbest) {
            tbest = t;
            std::memcpy(best, cand, sizeof best);
        }
        pf_set_tuning(c, best, PF_TUNE_LEN);
    };
    for (int sweep = 0; sweep < 2; ++sweep) {
        for (int slot : {0, 1, 2, 3, 37}) {
            const int cands[5] = {1, 2, 4, 8, 16};
            for (int v : cands) {
                std::memcpy(cfg, best, sizeof cfg);
                cfg[slot] = v;
                trial(cfg);
            }
        }
        // fused or staged FP32 x passes
        for (int v : {0, 1}) {
            std::memcpy(cfg, best, sizeof cfg);
            cfg[39] = v;
            trial(cfg);
        }
        // fused x passes with two shared buffers or one (in place)
        if (c->fp32)
            for (int v : {0, 1}) {
                std::memcpy(cfg, best, sizeof cfg);
                cfg[42] = v;
                trial(cfg);
            }
        // real fields of the right-hand-side x pass read from global or staged
        if (c->fp32 && c->ph.elastic)
            for (int v : {0, 1}) {
                std::memcpy(cfg, best, sizeof cfg);
                cfg[41] = v;
                trial(cfg);
            }
        // elastic pass with the fused stage, with every stage over the three
        // fields, or as a three-CTA cluster (FP32)
        if (c->ph.elastic && !c->inhom) {
            // each form at several tile widths: the best width depends on the
            // form (registers and shared memory per column differ)
            for (int v : {0, 1})
                for (int tx : {16, 8, 4}) {
                    std::memcpy(cfg, best, sizeof cfg);
                    cfg[40] = v;
                    cfg[2] = tx;
                    trial(cfg);
                }
            // the cluster form with its own tile widths (16 or 8 columns)
            if (c->fp32)
                for (int tx : {16, 8}) {
                    std::memcpy(cfg, best, sizeof cfg);
                    cfg[40] = 2;
                    cfg[2] = tx;
                    trial(cfg);
                }
        }
        // compiled plans of length nz for the fused elastic pass, or none (-1)
        for (int pid = -1; pid <= compiled_plan_count(); ++pid) {
            if (pid > 0 && compiled_plan_len(pid) != c->g.nz) continue;
            std::memcpy(cfg, best, sizeof cfg);
            cfg[38] = pid;
            trial(cfg);
        }
        const int ns[3] = {c->g.nx, c->g.ny, c->g.nz};
        for (int a = 0; a < 3; ++a) {
            for (const auto& ord : radix_orders(ns[a], 12)) {
                std::memcpy(cfg, best, sizeof cfg);
                int* r = cfg + 4 + 11 * a;
                r[0] = (int)ord.size();
                for (int s = 0; s < kMaxRadices; ++s) r[1 + s] = s < (int)ord.size() ? ord[s] : 0;
                trial(cfg);
            }
        }
    }
    pf_set_tuning(c, best, PF_TUNE_LEN);
    if (ms_after) *ms_after = tbest;
    return check_launch(c, "pf_autotune");
}

static const char* kKernelNames[PF_NKERNELS] = {"z_stage_solve_ifft", "y_fft", "x_c2r_physics1_r2c",
                                                 "x_c2r_physics2_r2c", "z_elastic_contraction", "z_fft_scale_fE",
                                                 "z_step_completion_lte", "x_c2r_wrms", "wrms_reduce",
                                                 "stage_pointwise", "z_ifft"};

const char* pf_kernel_name(int kind) { return (kind >= 0 && kind < PF_NKERNELS) ? kKernelNames[kind] : "?"; }

int pf_profile_enable(pf_ctx* c, int on) {
    if (!c) return fail(c, PF_EINVAL, "pf_profile_enable: NULL context");
    c->prof_on = on != 0;
    c->prof_recs.clear();
    c->prof_next = 0;
    return PF_OK;
}

int pf_profile_read(pf_ctx* c, double* ms, double* bytes, long long* launches) {
    if (!c) return fail(c, PF_EINVAL, "pf_profile_read: NULL context");
    cudaSetDevice(c->dev);
    PF_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int k = 0; k < PF_NKERNELS; ++k) {
        if (ms) ms[k] = 0.0;
        if (bytes) bytes[k] = 0.0;
        if (launches) launches[k] = 0;
    }
    for (const auto& r : c->prof_recs) {
        float t = 0.f;
        PF_CUDA(c, cudaEventElapsedTime(&t, r.e0, r.e1));
        if (ms) ms[r.kind] += t;
        if (bytes) bytes[r.kind] += r.bytes;
        if (launches) launches[r.kind] += 1;
    }
    c->prof_recs.clear();
    c->prof_next = 0;
    return PF_OK;
}

int pf_get_attempts(pf_ctx* c, double* buf, int max_attempts) {
    if (!c) return fail(c, PF_EINVAL, "pf_get_attempts: NULL context");
    const int n = (int)(c->attempts.size() / 4);
    if (buf) {
        const int m = n < max_attempts ? n : max_attempts;
        std::memcpy(buf, c->attempts.data(), (size_t)m * 4 * sizeof(double));
    }
    return n;
}

}  // extern "C"
