// Fused x passes (FP32 compute type): packed real transforms along x with the
// real-space physics between them, organised so that the physics runs in the
// registers of the threads that finish the inverse transform and start the
// forward one.
//
// The forward transform of a line uses the radix order Fwd = (RM, ...); the
// inverse runs it reversed, so its last stage (radix RM, sub-transform size
// M = N/RM) leaves butterfly j holding the elements x = j + M t (t < RM) --
// exactly the inputs of butterfly j of the forward first stage.  One thread
// per (row pair, j) therefore takes the last inverse stage of every input
// field, evaluates the physics at its RM positions of both rows, and applies
// the first forward stage to every output field without a shared-memory
// round trip.  The C2R packing of two real rows into one complex line is
// folded into the first inverse stage (read straight from the staged
// half-spectrum rows), the R2C unpacking into the store.  Stages ping-pong
// between two shared-memory tiles of skewed lines.
#pragma once
#include "pf_xpass.cuh"

namespace pf {

// XF_PHYS2_STG: XF_PHYS2 with the stored real fields the physics reads
// copied into shared memory (cp.async) together with the input rows, so that
// the physics does not wait on global loads
enum XFMode { XF_PHYS1_H = 0, XF_PHYS1_RHS = 1, XF_PHYS2 = 2, XF_WRMS = 3, XF_PHYS2_STG = 4 };
template <int MODE>
struct XFIO {
    static constexpr bool PHYS2 = MODE == XF_PHYS2 || MODE == XF_PHYS2_STG;
    static constexpr int FIN = PHYS2 ? 3 : 4;  // input lines per row pair
    static constexpr int FOUT = MODE == XF_WRMS ? 0 : (MODE == XF_PHYS1_H ? 3 : 4);
};

// stages of a radix list, sub-transform size growing from NS: cur -> oth,
// then the pointers swap (the result is in cur)
template <int SIGN, int N, int NS, typename T2>
__device__ __forceinline__ void xf_run(T2*&, T2*&, int, const T2*, Radices<>) {}
template <int SIGN, int N, int NS, typename T2, int R, int... Rest>
__device__ __forceinline__ void xf_run(T2*& cur, T2*& oth, int nl, const T2* tw, Radices<R, Rest...>) {
    fft_stage_fixed<R, SIGN, N, NS>(cur, oth, nl, skewed_len(N), tw);
    __syncthreads();
    T2* t = cur;
    cur = oth;
    oth = t;
    xf_run<SIGN, N, NS * R>(cur, oth, nl, tw, Radices<Rest...>{});
}

// In-place stage of NL skewed lines (one shared buffer): every job's R
// inputs are loaded into registers, the CTA synchronises, then the
// butterflies are formed and stored, and the CTA synchronises again.
template <int R, int SIGN, int N, int NS, int NL, int NT, typename T2>
__device__ __forceinline__ void xf_stage_inplace(T2* S, const T2* __restrict__ tw) {
    constexpr int M = N / R, TWS = N / (NS * R), JOBS = NL * M, JPT = (JOBS + NT - 1) / NT, LS = N + N / 16;
    T2 v[JPT][R];
#pragma unroll
    for (int u = 0; u < JPT; ++u) {
        const int idx = threadIdx.x + u * NT;
        if (JOBS % NT == 0 || idx < JOBS) {
            const int line = idx / M, j = idx - line * M;
            const T2* s = S + line * LS;
            if constexpr (M % 16 == 0) {
                // skew(j + t M) = skew(j) + t (M + M/16)
                const T2* sj = s + skew<true>(j);
#pragma unroll
                for (int t = 0; t < R; ++t) v[u][t] = sj[t * (M + M / 16)];
            } else {
#pragma unroll
                for (int t = 0; t < R; ++t) v[u][t] = s[skew<true>(j + t * M)];
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < JPT; ++u) {
        const int idx = threadIdx.x + u * NT;
        if (JOBS % NT == 0 || idx < JOBS) {
            const int line = idx / M, j = idx - line * M;
            const int jq = j / NS, k = j - jq * NS;
            if constexpr (NS > 1) apply_twiddles<R, SIGN>(v[u], tw, k * TWS);
            Bfly<R, SIGN, T2>::run(v[u]);
            T2* d = S + line * LS;
            const int a = jq * NS * R;  // outputs at a + k + t NS
            if constexpr ((NS * R) % 16 == 0 && NS % 16 == 0) {
                T2* dk = d + skew<true>(a) + skew<true>(k);
#pragma unroll
                for (int t = 0; t < R; ++t) dk[t * (NS + NS / 16)] = v[u][t];
            } else if constexpr ((NS * R) % 16 == 0 && 16 % NS == 0) {
                // k + t NS crosses a 16-block boundary only at multiples of 16
                T2* dk = d + skew<true>(a) + k;
#pragma unroll
                for (int t = 0; t < R; ++t) dk[t * NS + ((t * NS) >> 4)] = v[u][t];
            } else if constexpr (NS == 1 && 16 % R == 0) {
                // a = j R and a + t stay inside one 16-block
                T2* dk = d + skew<true>(a);
#pragma unroll
                for (int t = 0; t < R; ++t) dk[t] = v[u][t];
            } else {
#pragma unroll
                for (int t = 0; t < R; ++t) d[skew<true>(a + k + t * NS)] = v[u][t];
            }
        }
    }
    __syncthreads();
}
template <int SIGN, int N, int NS, int NL, int NT, typename T2>
__device__ __forceinline__ void xf_run_inplace(T2*, const T2*, Radices<>) {}
template <int SIGN, int N, int NS, int NL, int NT, typename T2, int R, int... Rest>
__device__ __forceinline__ void xf_run_inplace(T2* S, const T2* tw, Radices<R, Rest...>) {
    xf_stage_inplace<R, SIGN, N, NS, NL, NT>(S, tw);
    xf_run_inplace<SIGN, N, NS * R, NL, NT>(S, tw, Radices<Rest...>{});
}

template <class Fwd, int P>
struct XFShape {
    static constexpr int N = RadProd<Fwd>::value;
    static constexpr int RM = RadInfo<Fwd>::first;  // radix of the fused stages
    static constexpr int M = N / RM;                 // butterflies per line in the fused stages
    static constexpr int NT = P * M;                 // one thread per (row pair, butterfly)
    static_assert(NT % 32 == 0 && NT <= 1024, "whole warps, at most 1024 threads");
    static constexpr int LS = N + N / 16;            // skewed line stride
};

// INPL: one shared buffer, every stage in place (half the shared memory, so
// more CTAs per SM, for a barrier more per stage); registers bounded to 64 a
// thread so that the registers do not cap the CTAs per SM first
template <typename T, class Fwd, int P, int MODE, bool INPL>
__global__ void __launch_bounds__(XFShape<Fwd, P>::NT, INPL ? (65536 / (XFShape<Fwd, P>::NT * 64) > 0
                                                                     ? 65536 / (XFShape<Fwd, P>::NT * 64)
                                                                     : 1)
                                                              : 1)
    k_x_fused(Geo g, Phys ph, const float2* __restrict__ in,
                                                                  float2* __restrict__ out, float* __restrict__ R,
                                                                  const float* __restrict__ Rin,
                                                                  double* __restrict__ partials, float rt, float at) {
    PF_SKIP_INACTIVE(g);
    using T2 = float2;
    using Sh = XFShape<Fwd, P>;
    constexpr int N = Sh::N, RM = Sh::RM, M = Sh::M, NT = Sh::NT, LS = Sh::LS, NXH = N / 2 + 1;
    constexpr int FIN = XFIO<MODE>::FIN, FOUT = XFIO<MODE>::FOUT;
    using Inv = Reversed<Fwd>;
    constexpr int R1 = RadInfo<Inv>::first;  // first inverse stage
    extern __shared__ __align__(16) unsigned char smraw[];
    T2* A = reinterpret_cast<T2*>(smraw);
    T2* B = INPL ? A : A + P * 4 * LS;
    const int npairs = g.nz * g.ny / 2;
    const int rp0 = blockIdx.x * P;
    const long long NK = g.NK, N3 = g.N;
    const T2* tw = g.px.tw32;
    __shared__ double red[NT / 32 + 1];

    // 1. the raw half-spectrum rows of the input fields -> B (cp.async).  Raw
    //    row r = (rp FIN + f) 2 + (0: row y, 1: row y+1) goes to B + r NXH.
    //    NXH is odd and NK even, so row r starts 16-byte aligned in global and
    //    shared memory alike when r is even and one element later when r is
    //    odd: each row is NXH/2 16-byte copies from its first aligned element
    //    and one 8-byte copy of the element left over (the last or the first)
    {
        static_assert(NXH % 2 == 1, "odd half-spectrum rows");
        constexpr int NC = NXH / 2 + 1;  // copies per row: NXH/2 pairs and one single
        for (int e = threadIdx.x; e < P * FIN * 2 * NC; e += NT) {
            const int r = e / NC, c = e - r * NC;
            const int pf = r >> 1, rp = pf / FIN, f = pf - rp * FIN;
            const int head = r & 1;  // first element of the aligned pairs
            const int k = c < NXH / 2 ? head + 2 * c : (head ? 0 : NXH - 1);
            T2* dst = B + r * NXH + k;
            if (rp0 + rp < npairs) {
                const T2* src = in + (long long)f * NK + (2LL * (rp0 + rp) + head) * NXH + k;
                if (c < NXH / 2)
                    cp_async<16>(dst, src);
                else
                    cp_async<8>(dst, src);
            } else {
                dst[0] = T2{0.f, 0.f};
                if (c < NXH / 2) dst[1] = T2{0.f, 0.f};
            }
        }
    }
    // the real fields X, phi_v of the CTA's rows -> C ([row pair][field][2 rows][N]), 16-byte copies
    constexpr bool STG = MODE == XF_PHYS2_STG;
    float* C = reinterpret_cast<float*>(B + P * 4 * LS);
    if constexpr (STG) {
        constexpr int Q = N / 4;  // 16-byte chunks per row
        for (int e = threadIdx.x; e < P * 8 * Q; e += NT) {
            const int r = e / Q, q = e - r * Q;  // r = (rp 4 + f) 2 + (0: row y, 1: row y+1)
            const int rp = r >> 3, f = (r >> 1) & 3;
            if (rp0 + rp < npairs)
                cp_async<16>(C + 4 * e, Rin + f * N3 + (2LL * (rp0 + rp) + (r & 1)) * N + 4 * q);
            else
                reinterpret_cast<float4*>(C)[e] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    cp_async_wait_all();
    __syncthreads();
    // 2. first inverse stage (radix R1, no twiddles), packing Z = a + i b of
    //    the two rows' half spectra (Hermitian extension, imaginary parts of
    //    DC and Nyquist dropped): B -> A (in place: all loads, a barrier, the stores)
    {
        constexpr int M1 = N / R1, JOBS = P * FIN * M1, JPT = INPL ? (JOBS + NT - 1) / NT : 1;
        auto load = [&](int idx, T2* v) {
            const int line = idx / M1, j = idx - line * M1;
            const T2* ra = B + line * 2 * NXH;
            const T2* rb = ra + NXH;
#pragma unroll
            for (int t = 0; t < R1; ++t) {
                const int x = j + t * M1;
                const bool lo = x <= N / 2;
                const int k = lo ? x : N - x;
                T2 a = ra[k], b = rb[k];
                if (k == 0 || k == N / 2) {
                    a.y = 0.f;
                    b.y = 0.f;
                }
                v[t] = lo ? T2{a.x - b.y, a.y + b.x} : T2{a.x + b.y, b.x - a.y};
            }
        };
        auto store = [&](int idx, T2* v) {
            const int line = idx / M1, j = idx - line * M1;
            Bfly<R1, +1, T2>::run(v);
            T2* d = A + line * LS;
#pragma unroll
            for (int t = 0; t < R1; ++t) d[skew<true>(j * R1 + t)] = v[t];
        };
        if constexpr (INPL) {
            T2 v[JPT][R1];
#pragma unroll
            for (int u = 0; u < JPT; ++u)
                if (JOBS % NT == 0 || threadIdx.x + u * NT < JOBS) load(threadIdx.x + u * NT, v[u]);
            __syncthreads();
#pragma unroll
            for (int u = 0; u < JPT; ++u)
                if (JOBS % NT == 0 || threadIdx.x + u * NT < JOBS) store(threadIdx.x + u * NT, v[u]);
        } else {
            for (int idx = threadIdx.x; idx < JOBS; idx += NT) {
                T2 v[R1];
                load(idx, v);
                store(idx, v);
            }
        }
    }
    __syncthreads();
    T2* cur = A;
    T2* oth = B;
    // 3. inverse stages between the first and the last
    if constexpr (INPL)
        xf_run_inplace<+1, N, R1, P * FIN, NT>(cur, tw, typename PlanInner<Inv>::type{});
    else
        xf_run<+1, N, R1>(cur, oth, P * FIN, tw, typename PlanInner<Inv>::type{});
    // 4. fused: last inverse stage, physics, first forward stage
    const int rp = threadIdx.x / M, j = threadIdx.x - (threadIdx.x / M) * M;
    const bool valid = rp0 + rp < npairs;
    const long long row = 2LL * (rp0 + rp);
    T2 vin[FIN][RM];
#pragma unroll
    for (int f = 0; f < FIN; ++f) {
        const T2* src = cur + (rp * FIN + f) * LS;
#pragma unroll
        for (int t = 0; t < RM; ++t) vin[f][t] = src[skew<true>(j + t * M)];
        apply_twiddles<RM, +1>(vin[f], tw, j);  // NS = M: twiddle exponent j t
        Bfly<RM, +1, T2>::run(vin[f]);
    }
    if constexpr (MODE == XF_WRMS) {
        // sum of squares of the weighted error w_i LTE_i (weights from the
        // stored real-space y_{n-1}); compensated FP32 sum per thread, FP64
        // across threads and CTAs
        float sh = 0.f, sl = 0.f;
        if (valid) {
#pragma unroll
            for (int t = 0; t < RM; ++t) {
                const int x = j + t * M;
#pragma unroll
                for (int f = 0; f < FIN; ++f) {
                    const float* yr = Rin + f * N3 + row * N + x;
                    const float a = __fdividef(vin[f][t].x, __fmaf_rn(rt, fabsf(yr[0]), at));
                    const float b = __fdividef(vin[f][t].y, __fmaf_rn(rt, fabsf(yr[N]), at));
                    const DF s1 = df_two_sum(sh, __fmul_rn(a, a));
                    const DF s2 = df_two_sum(s1.h, __fmul_rn(b, b));
                    sh = s2.h;
                    sl = __fadd_rn(sl, __fadd_rn(s1.l, s2.l));
                }
            }
        }
        double acc = f2d_bits(sh) + f2d_bits(sl);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int i = 0; i < (NT + 31) / 32; ++i) s += red[i];
            partials[blockIdx.x] = s;
        }
        return;
    } else {
        const PhysT<float>& pt = ph.t32;
        T2 vout[FOUT][RM];
#pragma unroll
        for (int t = 0; t < RM; ++t) {
            const int x = j + t * M;
            float Xr[2], pr[2][3], er[2][3];
            if constexpr (XFIO<MODE>::PHYS2) {
#pragma unroll
                for (int f = 0; f < 4; ++f) {
                    float u0, u1;
                    if constexpr (STG) {
                        const float* c = C + ((rp * 4 + f) * 2) * N + x;
                        u0 = c[0];
                        u1 = c[N];
                    } else {
                        const float* b = Rin + f * N3 + row * N + x;
                        u0 = valid ? b[0] : 0.f;
                        u1 = valid ? b[N] : 0.f;
                    }
                    if (f == 0) {
                        Xr[0] = u0;
                        Xr[1] = u1;
                    } else {
                        pr[0][f - 1] = u0;
                        pr[1][f - 1] = u1;
                    }
                }
#pragma unroll
                for (int v = 0; v < 3; ++v) {
                    er[0][v] = vin[v][t].x;
                    er[1][v] = vin[v][t].y;
                }
            } else {
                Xr[0] = vin[0][t].x;
                Xr[1] = vin[0][t].y;
#pragma unroll
                for (int v = 0; v < 3; ++v) {
                    pr[0][v] = vin[1 + v][t].x;
                    pr[1][v] = vin[1 + v][t].y;
                    er[0][v] = 0.f;
                    er[1][v] = 0.f;
                }
                if (R && valid) {
#pragma unroll
                    for (int f = 0; f < 4; ++f) {
                        float* b = R + f * N3 + row * N + x;
                        b[0] = vin[f][t].x;
                        b[N] = vin[f][t].y;
                    }
                }
            }
            if constexpr (MODE == XF_PHYS1_H) {
#pragma unroll
                for (int v = 0; v < 3; ++v) vout[v][t] = T2{hfun(pr[0][v]), hfun(pr[1][v])};
            } else {
                float q[2], gv[2][3];
#pragma unroll
                for (int r = 0; r < 2; ++r) Pt::rhs<float, false>(pt, Xr[r], pr[r], er[r], q[r], gv[r]);
                vout[0][t] = T2{q[0], q[1]};
#pragma unroll
                for (int v = 0; v < 3; ++v) vout[1 + v][t] = T2{gv[0][v], gv[1][v]};
            }
        }
        if constexpr (INPL) __syncthreads();  // every input of the fused stage read before the stores
#pragma unroll
        for (int f = 0; f < FOUT; ++f) {
            Bfly<RM, -1, T2>::run(vout[f]);  // first forward stage: NS = 1, no twiddles
            T2* d = oth + (rp * FOUT + f) * LS;
#pragma unroll
            for (int t = 0; t < RM; ++t) d[skew<true>(j * RM + t)] = vout[f][t];
        }
        __syncthreads();
        {
            T2* t = cur;
            cur = oth;
            oth = t;
        }
        // 5. the remaining forward stages
        if constexpr (INPL)
            xf_run_inplace<-1, N, RM, P * FOUT, NT>(cur, tw, typename DropFirst<Fwd>::type{});
        else
            xf_run<-1, N, RM>(cur, oth, P * FOUT, tw, typename DropFirst<Fwd>::type{});
        // 6. R2C unpacking of the two rows of each line and the store
        for (int e = threadIdx.x; e < P * FOUT * NXH; e += NT) {
            const int line = e / NXH, k = e - line * NXH, lrp = line / FOUT, f = line - lrp * FOUT;
            if (rp0 + lrp >= npairs) continue;
            const T2 Zk = cur[line * LS + skew<true>(k)];
            const T2 Zm = cur[line * LS + skew<true>(k == 0 ? 0 : N - k)];
            const T2 a = T2{(Zk.x + Zm.x) * 0.5f, (Zk.y - Zm.y) * 0.5f};
            const T2 b = T2{(Zk.y + Zm.y) * 0.5f, (Zm.x - Zk.x) * 0.5f};
            T2* base = out + (long long)f * NK + (2LL * (rp0 + lrp)) * NXH + k;
            base[0] = a;
            base[NXH] = b;
        }
    }
}

// fused plans by line length (FP32): the first forward radix is small so the
// fused stage holds few values per field; P row pairs per CTA, chosen so that
// the CTA is a whole number of warps
template <int N>
struct XFPlan {
    static constexpr bool ok = false;
};
#define PF_XF_PLAN(N_, P_, ...)              \
    template <>                              \
    struct XFPlan<N_> {                      \
        static constexpr bool ok = true;     \
        static constexpr int P = P_;         \
        using Fwd = Radices<__VA_ARGS__>;    \
    };
PF_XF_PLAN(64, 16, 4, 16)
PF_XF_PLAN(96, 8, 4, 8, 3)
PF_XF_PLAN(120, 4, 3, 8, 5)
PF_XF_PLAN(128, 8, 4, 8, 4)
PF_XF_PLAN(160, 4, 4, 8, 5)
PF_XF_PLAN(192, 4, 4, 16, 3)
PF_XF_PLAN(256, 4, 4, 16, 4)
PF_XF_PLAN(640, 2, 5, 16, 8)
#undef PF_XF_PLAN

template <int N, int MODE, bool INPL>
static int launch_x_fused_k(const Geo& g, const Phys& ph, const void* in, void* out, void* R, const void* Rin,
                            double* partials, double rtol, double atol, cudaStream_t s) {
    using Pl = XFPlan<N>;
    using Sh = XFShape<typename Pl::Fwd, Pl::P>;
    const size_t sm = (INPL ? 1 : 2) * (size_t)Pl::P * 4 * Sh::LS * sizeof(float2) +
                      (MODE == XF_PHYS2_STG ? (size_t)Pl::P * 8 * N * sizeof(float) : 0);
    const int npairs = g.nz * g.ny / 2;
    const int nb = (npairs + Pl::P - 1) / Pl::P;
    auto k = k_x_fused<float, typename Pl::Fwd, Pl::P, MODE, INPL>;
    set_smem(k, sm);
    k<<<nb, Sh::NT, sm, s>>>(g, ph, reinterpret_cast<const float2*>(in), reinterpret_cast<float2*>(out),
                             reinterpret_cast<float*>(R), reinterpret_cast<const float*>(Rin), partials, (float)rtol,
                             (float)atol);
    return nb;
}

template <int N, int MODE>
static int launch_x_fused_n(const Geo& g, const Phys& ph, const void* in, void* out, void* R, const void* Rin,
                            double* partials, double rtol, double atol, cudaStream_t s) {
    return g.xf_inpl ? launch_x_fused_k<N, MODE, true>(g, ph, in, out, R, Rin, partials, rtol, atol, s)
                     : launch_x_fused_k<N, MODE, false>(g, ph, in, out, R, Rin, partials, rtol, atol, s);
}

template <int N>
static int launch_x_fused_modes(const Geo& g, const Phys& ph, int mode, const void* in, void* out, void* R,
                                const void* Rin, double* partials, double rtol, double atol, cudaStream_t s) {
    if constexpr (!XFPlan<N>::ok) {
        return 0;
    } else {
        switch (mode) {
            case XM_PHYS1:
                return ph.elastic ? launch_x_fused_n<N, XF_PHYS1_H>(g, ph, in, out, R, Rin, partials, rtol, atol, s)
                                  : launch_x_fused_n<N, XF_PHYS1_RHS>(g, ph, in, out, R, Rin, partials, rtol, atol, s);
            case XM_PHYS2:
                if (!ph.elastic) return 0;
                return g.xf_stg ? launch_x_fused_n<N, XF_PHYS2_STG>(g, ph, in, out, R, Rin, partials, rtol, atol, s)
                                : launch_x_fused_n<N, XF_PHYS2>(g, ph, in, out, R, Rin, partials, rtol, atol, s);
            case XM_WRMS: return launch_x_fused_n<N, XF_WRMS>(g, ph, in, out, R, Rin, partials, rtol, atol, s);
            default: return 0;
        }
    }
}

// the fused x pass for FP32 contexts where the line length has a fused plan;
// returns the number of CTAs launched, 0 if it does not apply
int launch_x_fused(const Geo& g, const Phys& ph, int mode, const void* in, void* out, void* R, const void* Rin,
                          double* partials, double rtol, double atol, cudaStream_t s) {
    // the obstacle barrier runs the staged passes (the fused ones carry only the double well)
    if (g.xf_off || ph.obst) return 0;
    switch (g.nx) {
        case 64: return launch_x_fused_modes<64>(g, ph, mode, in, out, R, Rin, partials, rtol, atol, s);
        case 96: return launch_x_fused_modes<96>(g, ph, mode, in, out, R, Rin, partials, rtol, atol, s);
        case 120: return launch_x_fused_modes<120>(g, ph, mode, in, out, R, Rin, partials, rtol, atol, s);
        case 128: return launch_x_fused_modes<128>(g, ph, mode, in, out, R, Rin, partials, rtol, atol, s);
        case 160: return launch_x_fused_modes<160>(g, ph, mode, in, out, R, Rin, partials, rtol, atol, s);
        case 192: return launch_x_fused_modes<192>(g, ph, mode, in, out, R, Rin, partials, rtol, atol, s);
        case 256: return launch_x_fused_modes<256>(g, ph, mode, in, out, R, Rin, partials, rtol, atol, s);
        case 640: return launch_x_fused_modes<640>(g, ph, mode, in, out, R, Rin, partials, rtol, atol, s);
        default: return 0;
    }
}

}  // namespace pf
