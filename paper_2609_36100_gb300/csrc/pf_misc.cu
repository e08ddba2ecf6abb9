// Pointwise and single-thread kernels: stage assembly without a transform,
// the FP32-bulk stage-assembly and step-completion streams, the diagonal
// implicit solve, lambda tables, the batch controller kernels, the
// deterministic reduction and the k-space free-energy sum.
#include "pf_common.cuh"

namespace pf {
// ---------------------------------------------------------------------------
// pointwise kernels (FP64)
// ---------------------------------------------------------------------------
__global__ void k_stage_pointwise(Geo g, Phys ph, const double2* __restrict__ y, StageTerms st, int fe32,
                                  double2* __restrict__ zout) {
    PF_SKIP_INACTIVE(g);
    if (y_swapped(g)) y = g.yother;
    const long long total = 4LL * g.NK;
    for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < total;
         gi += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(gi / g.NK);
        const long long r = gi % g.NK;
        const int kx = (int)(r % g.nxh);
        const int ky = (int)((r / g.nxh) % g.ny);
        const int kz = (int)(r / ((long long)g.nxh * g.ny));
        const double lam = lam_at(g, ph, f, gi, g.kx[kx], g.ky[ky], g.kz[kz]);
        double2 v = y[gi];
#pragma unroll
        for (int j = 0; j < kMaxStages; ++j) {
            if (j < st.n) {
                if ((st.mI >> j) & 1u) axpy(v, cI_of(st, j) * lam, st.z[j][gi]);
                if ((st.mE >> j) & 1u)
                    axpy(v, cE_of(st, j), fe32 ? load_f<float2>(st.f[j], gi) : load_f<double2>(st.f[j], gi));
            }
        }
        if (st.has_gamma) {
            const double q = st.qin ? st.qin[gi] : 1.0 / (1.0 - gamma_of(st) * lam);
            v.x *= q;
            v.y *= q;
        }
        zout[gi] = v;
    }
}

// FP32-bulk form: the double-float stage value of the z pass, without the
// transform (stages whose f^E no later stage or completion reads)
__global__ void k_stage_pointwise_df(Geo g, const double2* __restrict__ y, StageTerms st, float4* __restrict__ zout) {
    PF_SKIP_INACTIVE(g);
    if (y_swapped(g)) y = g.yother;
    const long long total = 4LL * g.NK;
    for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < total;
         gi += (long long)gridDim.x * blockDim.x)
        stage_value_df(g, st, y, gi, lam_row(g, gi), zout);
}

// FP32-bulk stage assembly, streaming: each element's loads all issued
// together (U elements per iteration for stages with few earlier terms), the
// double-float stage value z_i and its FP32 rounding (the input of the inverse
// z transform) written back.  Every array is read or written once.  DC: where
// the coefficients live (0: kernel parameters, 1: the batch's device copy);
// Idx: element index type.
//
// Element order: the grid strides over the wave vectors k, and each thread
// takes the four fields of its k (U at a time, their loads in flight
// together), so with shared phi rows (g.lam2) the lambda and q rows of the
// three phi fields are read from DRAM once and then hit in L1.
template <int MAXT, int U, int DC, typename Idx>
__global__ void __launch_bounds__(256) k_stage_assemble_df(Geo g, const double2* __restrict__ y, StageTerms st,
                                                           float4* __restrict__ zout, float2* __restrict__ W) {
    static_assert(4 % U == 0, "U divides the four fields");
    PF_SKIP_INACTIVE(g);
    if (y_swapped(g)) y = g.yother;
    const Idx nk = (Idx)g.NK;
    const Idx stride = (Idx)gridDim.x * blockDim.x;
    for (Idx k = (Idx)blockIdx.x * blockDim.x + threadIdx.x; k < nk; k += stride) {
#pragma unroll 1
        for (int f0 = 0; f0 < 4; f0 += U) {
            float2 r[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const Idx gi = (Idx)(f0 + u) * nk + k;
                const Idx ti = (g.lam2 && f0 + u > 0) ? nk + k : gi;
                r[u] = stage_value_df<MAXT, DC, Idx>(g, st, y, gi, ti, zout);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) W[(Idx)(f0 + u) * nk + k] = r[u];
        }
    }
}

// one wave of CTAs: every CTA resident at once, the grid-stride loop
// spreading the elements evenly (no partial last wave)
template <typename K>
static int resident_blocks(K kern, int threads) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0);
    return (sms > 0 ? sms : 152) * (per_sm > 0 ? per_sm : 1);
}

template <int MAXT, int U, int DC, typename Idx>
static void assemble_k(const Geo& g, const double2* y, const StageTerms& st, float4* z, float2* w, cudaStream_t s) {
    static int blocks = 0;  // per process: one device type
    if (blocks == 0) blocks = resident_blocks(k_stage_assemble_df<MAXT, U, DC, Idx>, 256);
    k_stage_assemble_df<MAXT, U, DC, Idx><<<blocks, 256, 0, s>>>(g, y, st, z, w);
}

template <int MAXT, int U>
static void assemble(const Geo& g, const double2* y, const StageTerms& st, float4* z, float2* w, cudaStream_t s) {
    // 32-bit indices while every index the loop forms (below 4 NK plus U
    // grid strides of at most a few million) stays below 2^32
    const bool idx32 = 4LL * g.NK <= (1LL << 32) - (1LL << 26);
    if (st.dc) {
        if (idx32)
            assemble_k<MAXT, U, 1, unsigned>(g, y, st, z, w, s);
        else
            assemble_k<MAXT, U, 1, long long>(g, y, st, z, w, s);
    } else {
        if (idx32)
            assemble_k<MAXT, U, 0, unsigned>(g, y, st, z, w, s);
        else
            assemble_k<MAXT, U, 0, long long>(g, y, st, z, w, s);
    }
}

void launch_stage_assemble(const Geo& g, const double2* y, const StageTerms& st, double2* zout, void* W,
                           cudaStream_t s) {
    float4* z = reinterpret_cast<float4*>(zout);
    float2* w = reinterpret_cast<float2*>(W);
    if (st.n == 0)
        assemble<0, 4>(g, y, st, z, w, s);
    else if (st.n <= 2)
        assemble<2, 2>(g, y, st, z, w, s);
    else if (st.n <= 5)
        assemble<5, 1>(g, y, st, z, w, s);
    else
        assemble<kMaxStages, 1>(g, y, st, z, w, s);
}

// FP32-bulk step completion, streaming: the new FP64 state and the FP32
// local error estimate of every element (the error's inverse z transform is a
// separate in-place pass).  Template arguments as in the stage assembly.
template <int MAXT, int DC, typename Idx>
__global__ void __launch_bounds__(256) k_step_complete_df(Geo g, const double2* __restrict__ y, StageTerms bt,
                                                          StageTerms dt, int want_lte, double2* __restrict__ ynew,
                                                          float2* __restrict__ W) {
    PF_SKIP_INACTIVE(g);
    if (y_swapped(g)) {
        double2* other = const_cast<double2*>(y);
        y = ynew;
        ynew = other;
    }
    // element order as in the stage assembly: the four fields of a k per thread
    const Idx nk = (Idx)g.NK;
    const Idx stride = (Idx)gridDim.x * blockDim.x;
    for (Idx k = (Idx)blockIdx.x * blockDim.x + threadIdx.x; k < nk; k += stride) {
#pragma unroll 1
        for (int f = 0; f < 4; ++f) {
            const Idx gi = (Idx)f * nk + k;
            const Idx ti = (g.lam2 && f > 0) ? nk + k : gi;
            const float2 e = final_value_df<MAXT, DC, Idx>(g, bt, dt, want_lte, y, gi, ti, ynew);
            if (want_lte) W[gi] = e;
        }
    }
}

template <int MAXT, int DC, typename Idx>
static void complete_k(const Geo& g, const double2* y, const StageTerms& bt, const StageTerms& dt, int want_lte,
                       double2* ynew, float2* w, cudaStream_t s) {
    static int blocks = 0;
    if (blocks == 0) blocks = resident_blocks(k_step_complete_df<MAXT, DC, Idx>, 256);
    k_step_complete_df<MAXT, DC, Idx><<<blocks, 256, 0, s>>>(g, y, bt, dt, want_lte, ynew, w);
}

template <int MAXT>
static void complete(const Geo& g, const double2* y, const StageTerms& bt, const StageTerms& dt, int want_lte,
                     double2* ynew, float2* w, cudaStream_t s) {
    const bool idx32 = 4LL * g.NK <= (1LL << 32) - (1LL << 26);
    if (bt.dc) {
        if (idx32)
            complete_k<MAXT, 1, unsigned>(g, y, bt, dt, want_lte, ynew, w, s);
        else
            complete_k<MAXT, 1, long long>(g, y, bt, dt, want_lte, ynew, w, s);
    } else {
        if (idx32)
            complete_k<MAXT, 0, unsigned>(g, y, bt, dt, want_lte, ynew, w, s);
        else
            complete_k<MAXT, 0, long long>(g, y, bt, dt, want_lte, ynew, w, s);
    }
}

void launch_step_complete(const Geo& g, const double2* y, const StageTerms& bt, const StageTerms& dt, int want_lte,
                          double2* ynew, void* W, cudaStream_t s) {
    float2* w = reinterpret_cast<float2*>(W);
    if (bt.n <= 6)
        complete<6>(g, y, bt, dt, want_lte, ynew, w, s);
    else
        complete<kMaxStages>(g, y, bt, dt, want_lte, ynew, w, s);
}

void launch_stage_pointwise(const Geo& g, const Phys& ph, const double2* y, const StageTerms& st, int fe_is_f32,
                            double2* zout, cudaStream_t s) {
    if (fe_is_f32)
        k_stage_pointwise_df<<<152 * 8, 256, 0, s>>>(g, y, st, reinterpret_cast<float4*>(zout));
    else
        k_stage_pointwise<<<152 * 8, 256, 0, s>>>(g, ph, y, st, 0, zout);
}

__global__ void k_solve(Geo g, Phys ph, double gamma, const double2* r, double2* z) {
    const long long total = 4LL * g.NK;
    for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < total;
         gi += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(gi / g.NK);
        const long long q = gi % g.NK;
        const int kx = (int)(q % g.nxh);
        const int ky = (int)((q / g.nxh) % g.ny);
        const int kz = (int)(q / ((long long)g.nxh * g.ny));
        const double den = 1.0 - gamma * lambda_k(ph, f, g.kx[kx], g.ky[ky], g.kz[kz]);
        const double2 v = r[gi];
        z[gi] = make_double2(v.x / den, v.y / den);
    }
}

void launch_solve(const Geo& g, const Phys& ph, double gamma, const double2* r, double2* z, cudaStream_t s) {
    k_solve<<<152 * 8, 256, 0, s>>>(g, ph, gamma, r, z);
}

__global__ void k_lambda_table(Geo g, Phys ph, double* __restrict__ lam, float2* __restrict__ lamdf) {
    const long long total = 4LL * g.NK;
    for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < total;
         gi += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(gi / g.NK);
        const long long q = gi % g.NK;
        const int kx = (int)(q % g.nxh);
        const int ky = (int)((q / g.nxh) % g.ny);
        const int kz = (int)(q / ((long long)g.nxh * g.ny));
        const double l = lambda_k(ph, f, g.kx[kx], g.ky[ky], g.kz[kz]);
        lam[gi] = l;
        if (lamdf && (!g.lam2 || f <= 1)) {  // shared phi rows: row 1 serves every phi field
            const float h = (float)l;
            lamdf[gi] = make_float2(h, (float)(l - (double)h));
        }
    }
}

// B_vq(k) / N in FP64, rounded to FP32, over kx in [0, nx/2], ky, kz in
// [0, n/2] (the kernel is even in each component for diagonal eigenstrains)
__global__ void k_btab(Geo g, Phys ph, float* __restrict__ tab) {
    const int hy = g.ny / 2 + 1, hz = g.nz / 2 + 1;
    const long long n = (long long)hz * hy * g.nxh;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int kx = (int)(i % g.nxh);
        const int ky = (int)((i / g.nxh) % hy);
        const int kz = (int)(i / ((long long)g.nxh * hy));
        double Bm[3][3];
        elastic_kernel<double>(ph.t64, g.kx[kx], g.ky[ky], g.kz[kz], Bm);
        const double s = g.invN;
        tab[0 * n + i] = (float)(Bm[0][0] * s);
        tab[1 * n + i] = (float)(Bm[0][1] * s);
        tab[2 * n + i] = (float)(Bm[0][2] * s);
        tab[3 * n + i] = (float)(Bm[1][1] * s);
        tab[4 * n + i] = (float)(Bm[1][2] * s);
        tab[5 * n + i] = (float)(Bm[2][2] * s);
    }
}

void launch_btab(const Geo& g, const Phys& ph, float* btab, cudaStream_t s) {
    k_btab<<<152 * 8, 256, 0, s>>>(g, ph, btab);
}

// the obstacle barrier's bound: real-space order parameters (fields 1-3 of a
// [4][N] FP64 array) clamped to [0, 1]
__global__ void k_clamp_phi(double* __restrict__ real, long long N) {
    for (long long i = N + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 4 * N;
         i += (long long)gridDim.x * blockDim.x)
        real[i] = fmin(1.0, fmax(0.0, real[i]));
}

void launch_clamp_phi(double* real, long long N, cudaStream_t s) { k_clamp_phi<<<152 * 8, 256, 0, s>>>(real, N); }

void launch_lambda_table(const Geo& g, const Phys& ph, double* lam, float2* lamdf, cudaStream_t s) {
    k_lambda_table<<<152 * 8, 256, 0, s>>>(g, ph, lam, lamdf);
}

// ---------------------------------------------------------------------------
// batch round kernels (one thread each, or a grid-stride copy)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void fill_coef(StageCoefDev& c, int n, const double* aI, const double* aE, double dt,
                                          double gam, double qgam) {
    for (int j = 0; j < kMaxStages; ++j) {
        const double ci = j < n ? dt * aI[j] : 0.0;
        const double ce = j < n ? dt * aE[j] : 0.0;
        c.cI[j] = ci;
        c.cE[j] = ce;
        const float h = (float)ce;
        c.cEh[j] = h;
        c.cEl[j] = (float)(ce - (double)h);
        const float hi = (float)ci;
        c.cIh[j] = hi;
        c.cIl[j] = (float)(ci - (double)hi);
    }
    c.gamma = gam;
    c.qgamma = qgam;
    c.gh = (float)gam;
    c.gl = (float)(gam - (double)c.gh);
    c.qgh = (float)qgam;
    c.qgl = (float)(qgam - (double)c.qgh);
}

// step size of this round's attempt (clipped to t_final) and the stage /
// completion coefficients built from it, as the host driver builds them
__global__ void k_batch_prep(BatchConst bc, MemberCtl* __restrict__ ctl, StageCoefDev* __restrict__ coef) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    MemberCtl& m = *ctl;
    if (!m.active) return;
    const double dt = fmin(m.h, bc.t_final - m.t);
    m.dt = dt;
    for (int i = 0; i < bc.s; ++i)
        fill_coef(coef[i], i, bc.AI[i], bc.AE[i], dt, dt * bc.AI[i][i], dt * bc.gdiag);
    double dI[kMaxStages], dE[kMaxStages];
    for (int j = 0; j < kMaxStages; ++j) {
        dI[j] = bc.embedded ? bc.bI[j] - bc.btI[j] : 0.0;
        dE[j] = bc.embedded ? bc.bE[j] - bc.btE[j] : 0.0;
    }
    fill_coef(coef[bc.s], bc.s, bc.bI, bc.bE, dt, 0.0, 0.0);
    fill_coef(coef[bc.s + 1], bc.s, dI, dE, dt, 0.0, 0.0);
}

// accept / reject and the next step size (same PI rule as the host driver)
__global__ void k_batch_ctl(BatchConst bc, MemberCtl* __restrict__ ctl, const double* __restrict__ wsum, double scale) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    MemberCtl& m = *ctl;
    m.accepted_now = 0;
    if (!m.active) return;
    const double e = bc.embedded ? sqrt(wsum[0] * scale) : 0.0;
    m.e_last = e;
    m.n_rhs += bc.nrhs;
    const bool ok = isfinite(e) && e <= 1.0;
    const double h = m.dt;
    double hn;
    if (ok) {
        m.t += h;
        m.n_acc += 1;
        m.nrej = 0;
        m.accepted_now = 1;
        m.ypar ^= 1;
        if (bc.embedded) {
            const double ee = e < 1e-10 ? 1e-10 : e;
            double eta = bc.safety * pow(ee, -bc.k1 / bc.q) * pow(m.e_prev, bc.k2 / bc.q);
            const double cap = m.after_reject ? 1.0 : bc.eta_max;
            eta = fmin(cap, fmax(bc.eta_min, eta));
            m.e_prev = ee;
            m.after_reject = 0;
            hn = h * eta;
        } else {
            hn = bc.h0;
        }
    } else {
        m.n_rej += 1;
        if (++m.nrej > bc.max_rejects) {
            m.status = isfinite(e) ? -5 : -4;  // PF_ESTEPFAIL / PF_ENONFINITE
            m.active = 0;
            return;
        }
        m.after_reject = 1;
        hn = isfinite(e) ? h * fmax(bc.eta_rej, bc.safety * pow(e, -1.0 / bc.q)) : h * 0.25;
    }
    m.h = fmin(fmax(hn, bc.h_min), bc.h_max);
    if (!(m.t < bc.t_final * (1 - 1e-14))) m.active = 0;
}


// Device-looped ensemble graph (a WHILE node around one round of every
// member, each member's round under an IF node).  The gate opens a member's
// IF node only while it is live; the loop condition is "some member live",
// with a round cap so that the loop always ends.  One thread each: calls
// that set one conditional handle must not race.
__global__ void k_batch_gate(const MemberCtl* __restrict__ ctl, const cudaGraphConditionalHandle* __restrict__ hif,
                             int n) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int m = 0; m < n; ++m) cudaGraphSetConditional(hif[m], ctl[m].active ? 1u : 0u);
}

__global__ void k_batch_more(const MemberCtl* __restrict__ ctl, int n, cudaGraphConditionalHandle hwhile,
                             unsigned long long* rounds, unsigned long long cap, int* capped) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int live = 0;
    for (int m = 0; m < n; ++m) live |= ctl[m].active;
    const unsigned long long r = ++*rounds;
    if (live && r >= cap) {
        *capped = 1;
        live = 0;
    }
    cudaGraphSetConditional(hwhile, live ? 1u : 0u);
}

cudaError_t add_batch_gate_node(cudaGraphNode_t* node, cudaGraph_t graph, const MemberCtl* ctl,
                                const cudaGraphConditionalHandle* hif, int n) {
    cudaKernelNodeParams kp{};
    void* args[] = {(void*)&ctl, (void*)&hif, (void*)&n};
    kp.func = (void*)k_batch_gate;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(32);
    kp.kernelParams = args;
    return cudaGraphAddKernelNode(node, graph, nullptr, 0, &kp);
}

cudaError_t add_batch_more_node(cudaGraphNode_t* node, cudaGraph_t graph, const cudaGraphNode_t* deps, size_t ndeps,
                                const MemberCtl* ctl, int n, cudaGraphConditionalHandle hwhile,
                                unsigned long long* rounds, unsigned long long cap, int* capped) {
    cudaKernelNodeParams kp{};
    void* args[] = {(void*)&ctl, (void*)&n, (void*)&hwhile, (void*)&rounds, (void*)&cap, (void*)&capped};
    kp.func = (void*)k_batch_more;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(32);
    kp.kernelParams = args;
    return cudaGraphAddKernelNode(node, graph, deps, ndeps, &kp);
}

void launch_batch_prep(const BatchConst& bc, MemberCtl* ctl, StageCoefDev* coef, cudaStream_t s) {
    k_batch_prep<<<1, 32, 0, s>>>(bc, ctl, coef);
}
void launch_batch_ctl(const BatchConst& bc, MemberCtl* ctl, const double* wrms_sum, double scale, cudaStream_t s) {
    k_batch_ctl<<<1, 32, 0, s>>>(bc, ctl, wrms_sum, scale);
}

// deterministic single-CTA reduction: out = sum(partials) * scale (FP64)
__global__ void k_reduce(const double* __restrict__ p, int n, double scale, double* out) {
    __shared__ double sh[1024];
    double a = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) a += p[i];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sh[0] * scale;
}

void launch_reduce(const double* partials, int n, double scale, double* out, cudaStream_t s) {
    k_reduce<<<1, 1024, 0, s>>>(partials, n, scale, out);
}

// *flag = 1 if any of the n FP64 words is NaN or infinite (all exponent bits
// set); the flag is cleared by the caller before the launch
__global__ void k_nonfinite(const unsigned long long* __restrict__ v, long long n, int* __restrict__ flag) {
    bool bad = false;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        bad |= ((v[i] >> 52) & 0x7ffull) == 0x7ffull;
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

void launch_nonfinite(const double* v, long long n, int* flag, cudaStream_t s) {
    k_nonfinite<<<152 * 8, 256, 0, s>>>(reinterpret_cast<const unsigned long long*>(v), n, flag);
}

// FMA throughput probe: eight independent FMA chains per thread (enough to
// hide the pipeline latency), `iters` rounds; the result is stored only if
// it equals a value it cannot reach, so nothing is optimised away.
template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(int iters, T b, T c, T* sink) {
    T a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = (T)(threadIdx.x + i) * (T)1e-3;
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = fma(a[i], b, c);
        }
    }
    T t = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) t += a[i];
    if (t == (T)-12345.678) *sink = t;
}

}  // namespace pf

extern "C" int pf_fma_peak(int precision, double* tflops) {
    using namespace pf;
    if (!tflops || (precision != 0 && precision != 1)) return -1;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -3;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    void* sink = nullptr;
    if (cudaMalloc(&sink, 16) != cudaSuccess) return -2;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int blocks = nsm * 8, threads = 256;
    // ~10^5 FMAs per thread in FP64 (the narrow pipe), ~5 10^6 in FP32
    const int iters = precision == 0 ? 800 : 40000;
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0, 0);
        if (precision == 0)
            k_fma_peak<double><<<blocks, threads>>>(iters, 0.999999, 1e-7, (double*)sink);
        else
            k_fma_peak<float><<<blocks, threads>>>(iters, 0.999999f, 1e-7f, (float*)sink);
        cudaEventRecord(e1, 0);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;  // the first launch is a warm-up
    }
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (err != cudaSuccess) return -3;
    const double flops = 2.0 * 8.0 * 16.0 * (double)iters * blocks * threads;
    *tflops = flops / (best * 1e-3) / 1e12;
    return 0;
}

namespace pf {

// k-space part of the free energy: sum_k w_k [ sum_v k.kappa_v.k |phi^_v|^2
//                                              + sum_vq B_vq Re(h^_v conj h^_q) ]
__global__ void k_energy_k(Geo g, Phys ph, const double2* __restrict__ y, const double2* __restrict__ hk,
                           double* partials) {
    __shared__ double red[8];
    double acc = 0.0;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < g.NK;
         r += (long long)gridDim.x * blockDim.x) {
        const int kx = (int)(r % g.nxh);
        const int ky = (int)((r / g.nxh) % g.ny);
        const int kz = (int)(r / ((long long)g.nxh * g.ny));
        const double w = (kx == 0 || (g.nx % 2 == 0 && kx == g.nx / 2)) ? 1.0 : 2.0;
        const double KX = g.kx[kx], KY = g.ky[ky], KZ = g.kz[kz];
        double s = 0.0;
        for (int v = 0; v < 3; ++v) {
            const double lam = lambda_k(ph, v + 1, KX, KY, KZ);  // -L k.kappa.k
            const double2 a = y[(long long)(v + 1) * g.NK + r];
            s += (-lam / ph.L) * (a.x * a.x + a.y * a.y);
        }
        if (ph.elastic) {
            double Bm[3][3];
            const PhysT<double>& pt = ph.t64;
            elastic_kernel<double>(pt, KX, KY, KZ, Bm);
            double2 h[3];
            for (int v = 0; v < 3; ++v) h[v] = hk[(long long)v * g.NK + r];
            for (int v = 0; v < 3; ++v)
                for (int q = 0; q < 3; ++q) s += Bm[v][q] * (h[v].x * h[q].x + h[v].y * h[q].y);
        }
        acc += w * s;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
        partials[blockIdx.x] = t;
    }
}

int energy_k_blocks(const Geo& g) { return 152 * 4; }

void launch_energy_k(const Geo& g, const Phys& ph, const double2* y, const double2* hk, double* partials,
                     cudaStream_t s) {
    k_energy_k<<<energy_k_blocks(g), 256, 0, s>>>(g, ph, y, hk, partials);
}


}  // namespace pf
