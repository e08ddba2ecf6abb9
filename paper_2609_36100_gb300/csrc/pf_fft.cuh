// Shared-memory mixed-radix (2,3,4,5,8,16) Stockham FFT used by every pass of
// the pseudospectral right-hand side.  A CTA transforms `nl` lines of length
// n held in shared memory; element e of line l sits at l*ls + e*es.  Stages
// ping-pong between two buffers; each butterfly reads R inputs strided by n/R,
// applies the twiddles exp(SIGN 2 pi i t k / (Ns R)) from an n-point table and
// writes R outputs strided by Ns (autosort, no bit reversal).
#pragma once
#include <cuda_runtime.h>

#include "pf_internal.h"

namespace pf {

constexpr int kColThreads = 256;  // threads of a column-pass CTA

template <typename T>
struct Cx;
template <>
struct Cx<double> {
    using t = double2;
};
template <>
struct Cx<float> {
    using t = float2;
};

template <typename T2>
__device__ __forceinline__ T2 cadd(T2 a, T2 b) { return T2{a.x + b.x, a.y + b.y}; }
template <typename T2>
__device__ __forceinline__ T2 csub(T2 a, T2 b) { return T2{a.x - b.x, a.y - b.y}; }
template <typename T2>
__device__ __forceinline__ T2 cmul(T2 a, T2 b) { return T2{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
// a * conj(b)
template <typename T2>
__device__ __forceinline__ T2 cmulc(T2 a, T2 b) { return T2{a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y}; }
// multiply by SIGN * i
template <int SIGN, typename T2>
__device__ __forceinline__ T2 mul_si(T2 a) {
    return SIGN > 0 ? T2{-a.y, a.x} : T2{a.y, -a.x};
}
template <typename T2, typename S>
__device__ __forceinline__ T2 cscale(T2 a, S s) { return T2{a.x * s, a.y * s}; }

// Butterfly constants (correctly rounded FP64): cos/sin of 2 pi/5, 4 pi/5, sin(pi/3), sqrt(2)/2.
#define PF_C1_5 0.30901699437494745
#define PF_C2_5 (-0.8090169943749475)
#define PF_S1_5 0.9510565162951535
#define PF_S2_5 0.5877852522924731
#define PF_S3 0.8660254037844386
#define PF_R2 0.7071067811865476
#define PF_C16 0.9238795325112867  // cos(pi/8)
#define PF_S16 0.3826834323650898  // sin(pi/8)

template <int R, int SIGN, typename T2>
struct Bfly;

template <int SIGN, typename T2>
struct Bfly<2, SIGN, T2> {
    __device__ __forceinline__ static void run(T2* v) {
        T2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <int SIGN, typename T2>
struct Bfly<4, SIGN, T2> {
    __device__ __forceinline__ static void run(T2* v) {
        T2 a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
        T2 c = cadd(v[1], v[3]), d = mul_si<SIGN>(csub(v[1], v[3]));
        v[0] = cadd(a, c);
        v[2] = csub(a, c);
        v[1] = cadd(b, d);
        v[3] = csub(b, d);
    }
};

template <int SIGN, typename T2>
struct Bfly<3, SIGN, T2> {
    __device__ __forceinline__ static void run(T2* v) {
        using T = decltype(v[0].x);
        T2 s = cadd(v[1], v[2]);
        T2 d = mul_si<SIGN>(cscale(csub(v[1], v[2]), (T)PF_S3));
        T2 m = csub(v[0], cscale(s, (T)0.5));
        v[0] = cadd(v[0], s);
        v[1] = cadd(m, d);
        v[2] = csub(m, d);
    }
};

template <int SIGN, typename T2>
struct Bfly<5, SIGN, T2> {
    __device__ __forceinline__ static void run(T2* v) {
        using T = decltype(v[0].x);
        const T c1 = (T)PF_C1_5, c2 = (T)PF_C2_5, s1 = (T)PF_S1_5, s2 = (T)PF_S2_5;
        T2 s = cadd(v[1], v[4]), d = csub(v[1], v[4]);
        T2 sp = cadd(v[2], v[3]), dp = csub(v[2], v[3]);
        T2 x0 = v[0];
        T2 a1 = T2{x0.x + c1 * s.x + c2 * sp.x, x0.y + c1 * s.y + c2 * sp.y};
        T2 a2 = T2{x0.x + c2 * s.x + c1 * sp.x, x0.y + c2 * s.y + c1 * sp.y};
        T2 b1 = mul_si<SIGN>(T2{s1 * d.x + s2 * dp.x, s1 * d.y + s2 * dp.y});
        T2 b2 = mul_si<SIGN>(T2{s2 * d.x - s1 * dp.x, s2 * d.y - s1 * dp.y});
        v[0] = cadd(x0, cadd(s, sp));
        v[1] = cadd(a1, b1);
        v[4] = csub(a1, b1);
        v[2] = cadd(a2, b2);
        v[3] = csub(a2, b2);
    }
};

template <int SIGN, typename T2>
struct Bfly<8, SIGN, T2> {
    __device__ __forceinline__ static void run(T2* v) {
        using T = decltype(v[0].x);
        T2 e[4] = {v[0], v[2], v[4], v[6]};
        T2 o[4] = {v[1], v[3], v[5], v[7]};
        Bfly<4, SIGN, T2>::run(e);
        Bfly<4, SIGN, T2>::run(o);
        const T r2 = (T)PF_R2;
        // w^m o_m with w = exp(SIGN i pi/4)
        T2 w1 = cscale(cadd(o[1], mul_si<SIGN>(o[1])), r2);
        T2 w2 = mul_si<SIGN>(o[2]);
        T2 w3 = cscale(csub(mul_si<SIGN>(o[3]), o[3]), r2);
        v[0] = cadd(e[0], o[0]);
        v[4] = csub(e[0], o[0]);
        v[1] = cadd(e[1], w1);
        v[5] = csub(e[1], w1);
        v[2] = cadd(e[2], w2);
        v[6] = csub(e[2], w2);
        v[3] = cadd(e[3], w3);
        v[7] = csub(e[3], w3);
    }
};

// 16 = 4 x 4: radix-4 DFTs over the stride-4 subsequences, twiddles
// w16^(n2 k1), radix-4 DFTs across them; w16 = exp(SIGN 2 pi i / 16)
template <int SIGN, typename T2>
struct Bfly<16, SIGN, T2> {
    __device__ __forceinline__ static T2 w16(T2 a, int m) {
        using T = decltype(a.x);
        const T c = (T)PF_C16, s = (T)PF_S16, r = (T)PF_R2;
        switch (m) {
            case 1: return cmul(a, T2{c, SIGN * s});
            case 2: return cmul(a, T2{r, SIGN * r});
            case 3: return cmul(a, T2{s, SIGN * c});
            case 4: return mul_si<SIGN>(a);
            case 6: return cmul(a, T2{-r, SIGN * r});
            case 9: return cmul(a, T2{-c, -SIGN * s});
            default: return a;
        }
    }
    __device__ __forceinline__ static void run(T2* v) {
        T2 A[4][4];
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) {
            T2 q[4] = {v[n2], v[4 + n2], v[8 + n2], v[12 + n2]};
            Bfly<4, SIGN, T2>::run(q);
#pragma unroll
            for (int k1 = 0; k1 < 4; ++k1) A[n2][k1] = w16(q[k1], n2 * k1);
        }
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            T2 q[4] = {A[0][k1], A[1][k1], A[2][k1], A[3][k1]};
            Bfly<4, SIGN, T2>::run(q);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = q[k2];
        }
    }
};

template <typename T2>
__device__ __forceinline__ const T2* twiddles(const AxisPlan& p);
template <>
__device__ __forceinline__ const double2* twiddles<double2>(const AxisPlan& p) { return p.tw64; }
template <>
__device__ __forceinline__ const float2* twiddles<float2>(const AxisPlan& p) { return p.tw32; }

// Exact unsigned division by a constant d >= 1 for numerators n with
// n * d < 2^32 (here n < 2^15, d <= 1024): q = (n * mul) >> 32 with
// mul = ceil(2^32 / d), computed on the host (see magic_u32).
struct FastDiv {
    unsigned d, mul;
    __device__ __forceinline__ FastDiv(unsigned dd, unsigned mm) : d(dd), mul(mm) {}
    __device__ __forceinline__ unsigned div(unsigned n) const { return d == 1 ? n : __umulhi(n, mul); }
};

// Skewed position of element i of a shared-memory line: one empty slot after
// every 16 elements.  The first Stockham stages write with stride R (and R*Ns)
// along a line; without the skew a warp's stores of 8- or 16-byte elements
// fall on a few banks (16-way conflicts for a radix-8 first stage), with it a
// radix-16 first stage is conflict-free and the (8, 8, 4) and (8, 4, 5) plans
// lose most of theirs (modelled over n = 64..256: 1.2x the conflict-free
// wavefront count for 8-byte elements, 1.03x for 16-byte ones).
template <bool SKEW>
__device__ __forceinline__ int skew(int i) {
    return SKEW ? i + (i >> 4) : i;
}
// line stride of n skewed elements
__host__ __device__ __forceinline__ int skewed_len(int n) { return n + (n >> 4); }

// One radix-R Stockham stage over all lines. LINE_FAST maps consecutive
// threads to consecutive lines (strided tiles, lines are contiguous columns);
// otherwise to consecutive butterflies of a line (contiguous x lines).
template <int R, int SIGN, bool LINE_FAST, int NL, bool SKEW = false, typename T2>
__device__ __forceinline__ void fft_stage(const T2* __restrict__ src, T2* __restrict__ dst, int n, int nl, int es,
                                          int ls, int Ns, const T2* __restrict__ tw, FastDiv divm, FastDiv divN,
                                          FastDiv divl) {
    const int m = n / R;
    const int total = nl * m;
    const int tws = n / (Ns * R);
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        int line, j;
        if constexpr (LINE_FAST) {
            if constexpr (NL > 0) {
                line = idx & (NL - 1);
                j = idx / NL;
            } else {
                j = (int)divl.div((unsigned)idx);
                line = idx - j * nl;
            }
        } else {
            line = (int)divm.div((unsigned)idx);
            j = idx - line * m;
        }
        const T2* s = src + line * ls;
        T2 v[R];
#pragma unroll
        for (int t = 0; t < R; ++t) v[t] = s[skew<SKEW>((j + t * m) * es)];
        const int jq = (int)divN.div((unsigned)j);
        const int k = j - jq * Ns;
        if (Ns > 1) {
            const int st = k * tws;
#pragma unroll
            for (int t = 1; t < R; ++t) {
                const T2 w = __ldg(tw + t * st);
                v[t] = SIGN < 0 ? cmul(v[t], w) : cmulc(v[t], w);
            }
        }
        Bfly<R, SIGN, T2>::run(v);
        const int base = jq * Ns * R + k;
        T2* d = dst + line * ls;
#pragma unroll
        for (int t = 0; t < R; ++t) d[skew<SKEW>((base + t * Ns) * es)] = v[t];
    }
}

// ---------------------------------------------------------------------------
// Compile-time plans for contiguous (skewed) lines: the length N, the radix
// order and each stage's sub-transform size NS are constants, so the line /
// butterfly split is a constant division and, wherever the skew allows, every
// shared-memory offset of a butterfly is an immediate from one per-thread
// base address (the generic stage spends about as many integer instructions
// on addressing as floating-point ones on the butterfly).
// ---------------------------------------------------------------------------
template <int... Rs>
struct Radices {};

// v[t] *= w^t (SIGN < 0) or conj(w)^t, w = tw[st], t = 1..R-1.  FP32 radix-8
// and radix-16 stages load w, w^2, w^4 (and w^8) from the table and form the
// other powers by at most three complex products (a few ulp, against the
// ulp-level rounding of the table itself), trading up to 11 dependent L1
// loads per butterfly for FMAs; FP64 stages (whose FMA pipe is the narrow
// one) load every power.
template <int R, int SIGN, typename T2>
__device__ __forceinline__ void apply_twiddles(T2* v, const T2* __restrict__ tw, int st) {
    auto mul = [](T2& x, T2 w) { x = SIGN < 0 ? cmul(x, w) : cmulc(x, w); };
    if constexpr (sizeof(T2) == 8 && (R == 8 || R == 16)) {
        // each power applied as soon as it is formed (few live registers)
        const T2 w1 = __ldg(tw + st), w2 = __ldg(tw + 2 * st), w4 = __ldg(tw + 4 * st);
        mul(v[1], w1);
        mul(v[2], w2);
        const T2 w3 = cmul(w2, w1);
        mul(v[3], w3);
        mul(v[4], w4);
        mul(v[5], cmul(w4, w1));
        mul(v[6], cmul(w4, w2));
        mul(v[7], cmul(w4, w3));
        if constexpr (R == 16) {
            const T2 w8 = __ldg(tw + 8 * st);
            mul(v[8], w8);
            mul(v[9], cmul(w8, w1));
            mul(v[10], cmul(w8, w2));
            mul(v[11], cmul(w8, w3));
            const T2 w12 = cmul(w8, w4);
            mul(v[12], w12);
            mul(v[13], cmul(w12, w1));
            mul(v[14], cmul(w12, w2));
            mul(v[15], cmul(w12, w3));
        }
    } else {
#pragma unroll
        for (int t = 1; t < R; ++t) mul(v[t], __ldg(tw + t * st));
    }
}

template <int R, int SIGN, int N, int NS, typename T2>
__device__ __forceinline__ void fft_stage_fixed(const T2* __restrict__ src, T2* __restrict__ dst, int nl, int ls,
                                                const T2* __restrict__ tw) {
    constexpr int M = N / R;           // butterflies per line
    constexpr int TWS = N / (NS * R);  // twiddle table stride of this stage
    static_assert(M * R == N, "radix does not divide the length");
    const int total = nl * M;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int line = idx / M, j = idx - line * M;
        const T2* s = src + line * ls;
        T2 v[R];
        if constexpr (M % 16 == 0) {
            // skew(j + t M) = skew(j) + t (M + M/16)
            const T2* sj = s + skew<true>(j);
#pragma unroll
            for (int t = 0; t < R; ++t) v[t] = sj[t * (M + M / 16)];
        } else {
#pragma unroll
            for (int t = 0; t < R; ++t) v[t] = s[skew<true>(j + t * M)];
        }
        const int jq = j / NS, k = j - jq * NS;
        if constexpr (NS > 1) {
            apply_twiddles<R, SIGN>(v, tw, k * TWS);
        }
        Bfly<R, SIGN, T2>::run(v);
        T2* d = dst + line * ls;
        const int a = jq * NS * R;  // output block start; outputs at a + k + t NS
        if constexpr ((NS * R) % 16 == 0 && NS % 16 == 0) {
            T2* dk = d + skew<true>(a) + skew<true>(k);
#pragma unroll
            for (int t = 0; t < R; ++t) dk[t * (NS + NS / 16)] = v[t];
        } else if constexpr ((NS * R) % 16 == 0 && 16 % NS == 0) {
            // k + t NS never crosses a 16-block boundary except at multiples of 16
            T2* dk = d + skew<true>(a) + k;
#pragma unroll
            for (int t = 0; t < R; ++t) dk[t * NS + ((t * NS) >> 4)] = v[t];
        } else if constexpr (NS == 1 && 16 % R == 0) {
            // a = j R and a + t stay inside one 16-block
            T2* dk = d + skew<true>(a);
#pragma unroll
            for (int t = 0; t < R; ++t) dk[t] = v[t];
        } else {
#pragma unroll
            for (int t = 0; t < R; ++t) d[skew<true>(a + k + t * NS)] = v[t];
        }
    }
}

template <int SIGN, int N, int NS, typename T2>
__device__ __forceinline__ T2* fft_fixed_run(T2* src, T2*, int, int, const T2*, Radices<>) {
    return src;
}

// Full transform of nl skewed lines with a compile-time plan; returns the
// buffer holding the result (synchronised).
template <int SIGN, int N, int NS, typename T2, int R, int... Rest>
__device__ __forceinline__ T2* fft_fixed_run(T2* src, T2* dst, int nl, int ls, const T2* tw, Radices<R, Rest...>) {
    fft_stage_fixed<R, SIGN, N, NS>(src, dst, nl, ls, tw);
    __syncthreads();
    return fft_fixed_run<SIGN, N, NS * R>(dst, src, nl, ls, tw, Radices<Rest...>{});
}

// Full transform of the lines in `a` (b is scratch).  Radix-16 stages are
// compiled in only with R16 (they raise the register count of the whole
// kernel); the launcher picks R16 from the plan (AxisPlan::has16).  Callers synchronise
// before; returns the buffer holding the result (synchronised).  NL > 0 fixes
// the line count at compile time (strided tiles of NL columns).
template <int SIGN, bool LINE_FAST, int NL = 0, bool SKEW = false, bool R16 = false, typename T2>
__device__ T2* fft_lines(T2* a, T2* b, const AxisPlan& p, int nl, int es, int ls, FastDiv divl = FastDiv(1, 0)) {
    const T2* tw = twiddles<T2>(p);
    T2* src = a;
    T2* dst = b;
    int Ns = 1;
    for (int s = 0; s < p.nst; ++s) {
        const int r = p.rad[s];
        const FastDiv dm((unsigned)(p.n / r), p.mulm[s]), dN((unsigned)Ns, p.mulN[s]);
        switch (r) {
            case 2: fft_stage<2, SIGN, LINE_FAST, NL, SKEW>(src, dst, p.n, nl, es, ls, Ns, tw, dm, dN, divl); break;
            case 3: fft_stage<3, SIGN, LINE_FAST, NL, SKEW>(src, dst, p.n, nl, es, ls, Ns, tw, dm, dN, divl); break;
            case 4: fft_stage<4, SIGN, LINE_FAST, NL, SKEW>(src, dst, p.n, nl, es, ls, Ns, tw, dm, dN, divl); break;
            case 5: fft_stage<5, SIGN, LINE_FAST, NL, SKEW>(src, dst, p.n, nl, es, ls, Ns, tw, dm, dN, divl); break;
            case 16:
                if constexpr (R16) fft_stage<16, SIGN, LINE_FAST, NL, SKEW>(src, dst, p.n, nl, es, ls, Ns, tw, dm, dN, divl);
                break;
            default: fft_stage<8, SIGN, LINE_FAST, NL, SKEW>(src, dst, p.n, nl, es, ls, Ns, tw, dm, dN, divl); break;
        }
        __syncthreads();
        T2* t = src;
        src = dst;
        dst = t;
        Ns *= r;
    }
    return src;
}

// ---------------------------------------------------------------------------
// Column-tile transform: TX lines ("columns", contiguous in global memory)
// of length n.  Stage 0 reads element (pos, col) through src(pos, col) --
// straight from global memory, with the pass's pointwise prologue fused --
// and the last stage hands each result to dst(pos, col, v); only the middle
// stages go through shared memory (layout [pos][TX]), ping-ponging between
// P and Q (P first).  Callers pick P/Q so that no stage reads and writes the
// same buffer.  With one stage and IN_PLACE (dst writes what src reads),
// results go through P first.
// ---------------------------------------------------------------------------
template <int R, int SIGN, int TX, typename T2, class Src, class Dst>
__device__ __forceinline__ void col_stage(int n, int Ns, FastDiv dN, const T2* __restrict__ in, T2* __restrict__ out,
                                          bool first, bool last, const T2* __restrict__ tw, Src& src, Dst& dst) {
    const int m = n / R;
    const int total = TX * m;
    const int tws = n / (Ns * R);
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int col = idx & (TX - 1);
        const int j = idx / TX;
        T2 v[R];
        if (first) {
#pragma unroll
            for (int t = 0; t < R; ++t) v[t] = src(j + t * m, col);
        } else {
#pragma unroll
            for (int t = 0; t < R; ++t) v[t] = in[(j + t * m) * TX + col];
        }
        const int jq = (int)dN.div((unsigned)j);
        const int k = j - jq * Ns;
        if (Ns > 1) {
            const int st = k * tws;
#pragma unroll
            for (int t = 1; t < R; ++t) {
                const T2 w = __ldg(tw + t * st);
                v[t] = SIGN < 0 ? cmul(v[t], w) : cmulc(v[t], w);
            }
        }
        Bfly<R, SIGN, T2>::run(v);
        const int base = jq * Ns * R + k;
        if (last) {
#pragma unroll
            for (int t = 0; t < R; ++t) dst(base + t * Ns, col, v[t]);
        } else {
#pragma unroll
            for (int t = 0; t < R; ++t) out[(base + t * Ns) * TX + col] = v[t];
        }
    }
}

//
// PRELOAD > 0: every element is first formed by src into P by a plain loop
// over the tile, unrolled PRELOAD times (one src inlined, its loads all
// independent and in flight together), and the stages then run from shared
// memory.  For heavy
// prologues (stage assembly from many global arrays) this keeps the memory
// parallelism and the register count of the transform independent of the
// prologue.
template <int SIGN, int TX, bool IN_PLACE = false, int PRELOAD = 0, bool R16 = false, typename T2, class Src,
          class Dst>
__device__ void fft_cols(const AxisPlan& p, T2* P, T2* Q, Src src, Dst dst) {
    const T2* tw = twiddles<T2>(p);
    const int n = p.n;
    if constexpr (PRELOAD > 0) {
        // unrolled PRELOAD times: the loads of several elements are in flight together
#pragma unroll PRELOAD
        for (int e = threadIdx.x; e < TX * n; e += blockDim.x) P[e] = src(e / TX, e & (TX - 1));
        __syncthreads();
        auto none = [](int, int) -> T2 { return T2{}; };
        const T2* in = P;
        T2* out = Q;
        int Ns = 1;
        for (int s = 0; s < p.nst; ++s) {
            const bool last = (s == p.nst - 1);
            const FastDiv dN((unsigned)Ns, p.mulN[s]);
            switch (p.rad[s]) {
                case 2: col_stage<2, SIGN, TX>(n, Ns, dN, in, out, false, last, tw, none, dst); break;
                case 3: col_stage<3, SIGN, TX>(n, Ns, dN, in, out, false, last, tw, none, dst); break;
                case 4: col_stage<4, SIGN, TX>(n, Ns, dN, in, out, false, last, tw, none, dst); break;
                case 5: col_stage<5, SIGN, TX>(n, Ns, dN, in, out, false, last, tw, none, dst); break;
                case 16:
                    if constexpr (R16) col_stage<16, SIGN, TX>(n, Ns, dN, in, out, false, last, tw, none, dst);
                    break;
                default: col_stage<8, SIGN, TX>(n, Ns, dN, in, out, false, last, tw, none, dst); break;
            }
            if (!last) __syncthreads();
            in = out;
            out = (out == P) ? Q : P;
            Ns *= p.rad[s];
        }
        return;
    }
    if (p.nst == 1 && IN_PLACE) {
        // single stage reading and writing the same global columns: stage
        // into P, then store
        auto toP = [&](int pos, int col, T2 v) { P[pos * TX + col] = v; };
        const FastDiv dN(1u, 0u);
        switch (p.rad[0]) {
            case 2: col_stage<2, SIGN, TX>(n, 1, dN, P, P, true, true, tw, src, toP); break;
            case 3: col_stage<3, SIGN, TX>(n, 1, dN, P, P, true, true, tw, src, toP); break;
            case 4: col_stage<4, SIGN, TX>(n, 1, dN, P, P, true, true, tw, src, toP); break;
            case 5: col_stage<5, SIGN, TX>(n, 1, dN, P, P, true, true, tw, src, toP); break;
            case 16:
                if constexpr (R16) col_stage<16, SIGN, TX>(n, 1, dN, P, P, true, true, tw, src, toP);
                break;
            default: col_stage<8, SIGN, TX>(n, 1, dN, P, P, true, true, tw, src, toP); break;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < TX * n; e += blockDim.x) dst(e / TX, e & (TX - 1), P[e]);
        return;
    }
    const T2* in = nullptr;
    T2* out = P;
    int Ns = 1;
    for (int s = 0; s < p.nst; ++s) {
        const bool first = (s == 0), last = (s == p.nst - 1);
        const FastDiv dN((unsigned)Ns, p.mulN[s]);
        switch (p.rad[s]) {
            case 2: col_stage<2, SIGN, TX>(n, Ns, dN, in, out, first, last, tw, src, dst); break;
            case 3: col_stage<3, SIGN, TX>(n, Ns, dN, in, out, first, last, tw, src, dst); break;
            case 4: col_stage<4, SIGN, TX>(n, Ns, dN, in, out, first, last, tw, src, dst); break;
            case 5: col_stage<5, SIGN, TX>(n, Ns, dN, in, out, first, last, tw, src, dst); break;
            case 16:
                if constexpr (R16) col_stage<16, SIGN, TX>(n, Ns, dN, in, out, first, last, tw, src, dst);
                break;
            default: col_stage<8, SIGN, TX>(n, Ns, dN, in, out, first, last, tw, src, dst); break;
        }
        if (!last) __syncthreads();
        in = out;
        out = (out == P) ? Q : P;
        Ns *= p.rad[s];
    }
}


// ---------------------------------------------------------------------------
// Plans compiled with a constant length and radix order (PID > 0), shared by
// the line (x) and column (y, z) transforms; any other plan runs the generic
// stages (PID 0).  The list holds the default plans of the grid sizes of the
// workloads (FP32 plans prefer radix 16, FP64 plans radix 8).
// ---------------------------------------------------------------------------
template <int PID>
struct FixedPlan {
    static constexpr int N = 0;
    using Rad = Radices<>;
};
#define PF_FIXED_PLAN(PID_, N_, ...)      \
    template <>                           \
    struct FixedPlan<PID_> {              \
        static constexpr int N = N_;      \
        using Rad = Radices<__VA_ARGS__>; \
    };
PF_FIXED_PLAN(1, 256, 16, 16)
PF_FIXED_PLAN(2, 256, 8, 8, 4)
PF_FIXED_PLAN(3, 128, 16, 8)
PF_FIXED_PLAN(4, 128, 8, 4, 4)
PF_FIXED_PLAN(5, 64, 16, 4)
PF_FIXED_PLAN(6, 64, 8, 8)
PF_FIXED_PLAN(7, 160, 8, 4, 5)
PF_FIXED_PLAN(8, 96, 8, 4, 3)
PF_FIXED_PLAN(9, 120, 8, 3, 5)
PF_FIXED_PLAN(10, 192, 16, 4, 3)
PF_FIXED_PLAN(11, 640, 16, 8, 5)
#undef PF_FIXED_PLAN
constexpr int kFixedPlans = 11;

template <int... Rs>
inline bool plan_is(const AxisPlan& p, int n, Radices<Rs...>) {
    const int r[] = {Rs...};
    if (p.n != n || p.nst != (int)sizeof...(Rs)) return false;
    for (int s = 0; s < p.nst; ++s)
        if (p.rad[s] != r[s]) return false;
    return true;
}

// length of compiled plan PID (0 for an unknown PID)
template <int PID = 1>
inline int fixed_plan_len(int pid) {
    if constexpr (PID > kFixedPlans) {
        return 0;
    } else {
        return pid == PID ? FixedPlan<PID>::N : fixed_plan_len<PID + 1>(pid);
    }
}

// PID of a plan (0: not compiled)
template <int PID = 1>
inline int fixed_plan_id(const AxisPlan& p) {
    if constexpr (PID > kFixedPlans) {
        return 0;
    } else {
        if (plan_is(p, FixedPlan<PID>::N, typename FixedPlan<PID>::Rad{})) return PID;
        return fixed_plan_id<PID + 1>(p);
    }
}

// Column stage with compile-time length, radix and sub-transform size: the
// same data movement as col_stage, with constant strides.
template <int R, int SIGN, int TX, int N, int NS, bool FIRST, bool LAST, typename T2, class Src, class Dst>
__device__ __forceinline__ void col_stage_fixed(const T2* __restrict__ in, T2* __restrict__ out,
                                                const T2* __restrict__ tw, Src& src, Dst& dst) {
    constexpr int M = N / R;
    constexpr int TWS = N / (NS * R);
    static_assert(M * R == N, "radix does not divide the length");
    for (int idx = threadIdx.x; idx < TX * M; idx += blockDim.x) {
        const int col = idx & (TX - 1);
        const int j = idx / TX;
        T2 v[R];
        if constexpr (FIRST) {
#pragma unroll
            for (int t = 0; t < R; ++t) v[t] = src(j + t * M, col);
        } else {
            const T2* p = in + j * TX + col;
#pragma unroll
            for (int t = 0; t < R; ++t) v[t] = p[t * M * TX];
        }
        const int jq = j / NS, k = j - jq * NS;
        if constexpr (NS > 1) {
            apply_twiddles<R, SIGN>(v, tw, k * TWS);
        }
        Bfly<R, SIGN, T2>::run(v);
        const int base = jq * NS * R + k;
        if constexpr (LAST) {
#pragma unroll
            for (int t = 0; t < R; ++t) dst(base + t * NS, col, v[t]);
        } else {
            T2* p = out + base * TX + col;
#pragma unroll
            for (int t = 0; t < R; ++t) p[t * NS * TX] = v[t];
        }
    }
}

template <int SIGN, int TX, int N, int NS, bool FIRST, typename T2, class Src, class Dst>
__device__ __forceinline__ void cols_fixed_run(const T2*, T2*, T2*, const T2*, Src&, Dst&, Radices<>) {}

// stages in order: stage 0 reads src (FIRST) or `in`, writes `out`; the
// middle stages ping-pong between out and other; the last hands results to dst
template <int SIGN, int TX, int N, int NS, bool FIRST, typename T2, class Src, class Dst, int R, int... Rest>
__device__ __forceinline__ void cols_fixed_run(const T2* in, T2* out, T2* other, const T2* tw, Src& src, Dst& dst,
                                               Radices<R, Rest...>) {
    constexpr bool LAST = sizeof...(Rest) == 0;
    col_stage_fixed<R, SIGN, TX, N, NS, FIRST, LAST>(in, out, tw, src, dst);
    if constexpr (!LAST) {
        __syncthreads();
        cols_fixed_run<SIGN, TX, N, NS * R, false>(out, other, out, tw, src, dst, Radices<Rest...>{});
    }
}

template <class Rad>
struct RadInfo;
template <int R, int... Rs>
struct RadInfo<Radices<R, Rs...>> {
    static constexpr int count = 1 + (int)sizeof...(Rs);
    static constexpr int first = R;
    static constexpr int last = RadInfo<Radices<Rs...>>::count == 0 ? R : RadInfo<Radices<Rs...>>::last;
};
template <>
struct RadInfo<Radices<>> {
    static constexpr int count = 0;
    static constexpr int first = 1;
    static constexpr int last = 1;
};

// largest radix of a list
template <class R>
struct RadMax;
template <>
struct RadMax<Radices<>> {
    static constexpr int value = 1;
};
template <int R, int... Rs>
struct RadMax<Radices<R, Rs...>> {
    static constexpr int value = R > RadMax<Radices<Rs...>>::value ? R : RadMax<Radices<Rs...>>::value;
};

// the radix order reversed: the inverse transform of a tile whose forward
// transform ended with radix R starts with radix R, so that the last forward
// stage and the first inverse stage see the same element positions
template <class A, class B>
struct RevCat;
template <int... Bs>
struct RevCat<Radices<>, Radices<Bs...>> {
    using type = Radices<Bs...>;
};
template <int A, int... As, int... Bs>
struct RevCat<Radices<A, As...>, Radices<Bs...>> {
    using type = typename RevCat<Radices<As...>, Radices<A, Bs...>>::type;
};
template <class R>
using Reversed = typename RevCat<R, Radices<>>::type;
// product of a radix list (the transform length)
template <class R>
struct RadProd;
template <int... Rs>
struct RadProd<Radices<Rs...>> {
    static constexpr int value = (Rs * ... * 1);
};

// the radices strictly between the first and the last of a list
template <class R>
struct DropFirst;
template <int A, int... Rs>
struct DropFirst<Radices<A, Rs...>> {
    using type = Radices<Rs...>;
};
template <class R>
struct PlanInner {
    using type = Reversed<typename DropFirst<Reversed<typename DropFirst<R>::type>>::type>;
};
template <int A>
struct PlanInner<Radices<A>> {
    using type = Radices<>;
};

// one radix-R stage of NF fields of the [f][pos][TX] tile S, in place: each
// thread first loads every butterfly it owns, the CTA synchronises, then the
// butterflies are computed and stored (and the CTA synchronises again)
template <int R, int SIGN, int TX, int N, int NS, int NF, int NT, typename T2>
__device__ __forceinline__ void tile_stage_inplace(T2* S, const T2* __restrict__ tw) {
    constexpr int M = N / R, JOBS = NF * TX * M, JPT = (JOBS + NT - 1) / NT, TWS = N / (NS * R);
    T2 v[JPT][R];
#pragma unroll
    for (int u = 0; u < JPT; ++u) {
        const int idx = threadIdx.x + u * NT;
        if (JOBS % NT == 0 || idx < JOBS) {
            const int f = idx / (TX * M), r = idx - f * (TX * M), col = r % TX, j = r / TX;
            const T2* src = S + f * (N * TX) + j * TX + col;
#pragma unroll
            for (int t = 0; t < R; ++t) v[u][t] = src[t * M * TX];
        }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < JPT; ++u) {
        const int idx = threadIdx.x + u * NT;
        if (JOBS % NT == 0 || idx < JOBS) {
            const int f = idx / (TX * M), r = idx - f * (TX * M), col = r % TX, j = r / TX;
            const int jq = j / NS, k = j - jq * NS;
            if constexpr (NS > 1) apply_twiddles<R, SIGN>(v[u], tw, k * TWS);
            Bfly<R, SIGN, T2>::run(v[u]);
            T2* dst = S + f * (N * TX) + (jq * NS * R + k) * TX + col;
#pragma unroll
            for (int t = 0; t < R; ++t) dst[t * NS * TX] = v[u][t];
        }
    }
    __syncthreads();
}

// Column transform of a compile-time plan with one shared buffer: stage 0
// reads global memory (src) into S, the middle stages run in place through
// registers (tile_stage_inplace), the last stage hands results to dst.
template <int SIGN, int TX, int N, int NS, bool FIRST, typename T2, class Src, class Dst>
__device__ __forceinline__ void cols_fixed_run_1buf(T2*, const T2*, Src&, Dst&, Radices<>) {}
template <int SIGN, int TX, int N, int NS, bool FIRST, typename T2, class Src, class Dst, int R, int... Rest>
__device__ __forceinline__ void cols_fixed_run_1buf(T2* S, const T2* tw, Src& src, Dst& dst, Radices<R, Rest...>) {
    constexpr bool LAST = sizeof...(Rest) == 0;
    if constexpr (FIRST || LAST) {
        col_stage_fixed<R, SIGN, TX, N, NS, FIRST, LAST>(S, S, tw, src, dst);
        if constexpr (!LAST) __syncthreads();
    } else {
        tile_stage_inplace<R, SIGN, TX, N, NS, 1, kColThreads>(S, tw);
    }
    cols_fixed_run_1buf<SIGN, TX, N, NS * R, false>(S, tw, src, dst, Radices<Rest...>{});
}

// fft_cols with the compile-time plan PID (same contract)
template <int SIGN, int TX, bool IN_PLACE, int PRELOAD, int PID, typename T2, class Src, class Dst>
__device__ void fft_cols_fixed(const AxisPlan& p, T2* P, T2* Q, Src src, Dst dst) {
    constexpr int N = FixedPlan<PID>::N;
    using Rad = typename FixedPlan<PID>::Rad;
    const T2* tw = twiddles<T2>(p);
    if constexpr (PRELOAD > 0) {
        // unrolled PRELOAD times: the loads of several elements are in flight together
#pragma unroll PRELOAD
        for (int e = threadIdx.x; e < TX * N; e += blockDim.x) P[e] = src(e / TX, e & (TX - 1));
        __syncthreads();
        auto none = [](int, int) -> T2 { return T2{}; };
        cols_fixed_run<SIGN, TX, N, 1, false>(P, Q, P, tw, none, dst, Rad{});
    } else if constexpr (IN_PLACE && RadInfo<Rad>::count == 1) {
        auto toP = [&](int pos, int col, T2 v) { P[pos * TX + col] = v; };
        col_stage_fixed<RadInfo<Rad>::first, SIGN, TX, N, 1, true, true>(P, P, tw, src, toP);
        __syncthreads();
        for (int e = threadIdx.x; e < TX * N; e += blockDim.x) dst(e / TX, e & (TX - 1), P[e]);
    } else {
        cols_fixed_run<SIGN, TX, N, 1, true>(static_cast<const T2*>(nullptr), P, Q, tw, src, dst, Rad{});
    }
}

// column transform with the compile-time plan PID, or the generic stages;
// ONEBUF: a compiled plan of three or more stages uses only P (its middle
// stages in place; the caller allocates one buffer, see col_buffers)
template <int SIGN, int TX, bool IN_PLACE, int PRELOAD, bool R16, int PID, bool ONEBUF = false, typename T2,
          class Src, class Dst>
__device__ __forceinline__ void cols_fft(const AxisPlan& p, T2* P, T2* Q, Src src, Dst dst) {
    if constexpr (PID > 0) {
        if constexpr (ONEBUF && PRELOAD == 0 && RadInfo<typename FixedPlan<PID>::Rad>::count >= 3) {
            cols_fixed_run_1buf<SIGN, TX, FixedPlan<PID>::N, 1, true>(P, twiddles<T2>(p), src, dst,
                                                                      typename FixedPlan<PID>::Rad{});
        } else {
            fft_cols_fixed<SIGN, TX, IN_PLACE, PRELOAD, PID>(p, P, Q, src, dst);
        }
    } else {
        fft_cols<SIGN, TX, IN_PLACE, PRELOAD, R16>(p, P, Q, src, dst);
    }
}

// shared-memory buffers of a column pass of the compute type T at tile
// width tx: one when the transform has at most two stages or runs a compiled
// plan (FP32, tile width 8 or 16), else two
template <typename T>
inline int col_buffers(const AxisPlan& p, int tx) {
    if (p.nst <= 2) return 1;
    const bool compiled = sizeof(T) == 4 && (tx == 8 || tx == 16) && fixed_plan_id(p) > 0;
    return compiled ? 1 : 2;
}

}  // namespace pf
