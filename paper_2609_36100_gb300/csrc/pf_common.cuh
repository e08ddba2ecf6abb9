// Device helpers shared by the pass kernels of the pseudospectral ImEx-ARK
// right-hand side: complex/double-float arithmetic, model constants in the
// compute type, wave numbers, tile-width choice, the FP32-bulk stage
// combination and the elastic Green's tensor.
#pragma once
#include <cstdio>
#include <type_traits>

#include "pf_fft.cuh"
#include "pf_internal.h"

namespace pf {

constexpr int kThreads = 256;

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
// lambda(k) of field f: -2 A^m M k^2 (X), -L k.kappa_v.k (phi_v); FP64.
// Isotropic gradient tensors reduce to lamc[f] * k^2.
__device__ __forceinline__ double lambda_k(const Phys& ph, int f, double kx, double ky, double kz) {
    const double k2 = kx * kx + ky * ky + kz * kz;
    if (f == 0 || ph.kap_iso) return ph.lamc[f] * k2;
    const double* K = ph.kap[f - 1];
    double kk = K[0] * kx * kx + K[1] * ky * ky + K[2] * kz * kz;
    kk += 2.0 * (K[3] * ky * kz + K[4] * kx * kz + K[5] * kx * ky);
    return -ph.L * kk;
}

template <typename T2>
__device__ __forceinline__ double2 to_d2(T2 a) { return make_double2((double)a.x, (double)a.y); }
template <typename T2>
__device__ __forceinline__ T2 from_d2(double2 a);
template <>
__device__ __forceinline__ double2 from_d2<double2>(double2 a) { return a; }
template <>
__device__ __forceinline__ float2 from_d2<float2>(double2 a) { return make_float2((float)a.x, (float)a.y); }

// stage coefficients: kernel parameters, or the batch member's device copy
__device__ __forceinline__ double cI_of(const StageTerms& st, int j) { return st.dc ? st.dc->cI[j] : st.cI[j]; }
__device__ __forceinline__ double cE_of(const StageTerms& st, int j) { return st.dc ? st.dc->cE[j] : st.cE[j]; }
__device__ __forceinline__ float cEh_of(const StageTerms& st, int j) { return st.dc ? st.dc->cEh[j] : st.cEh[j]; }
__device__ __forceinline__ float cEl_of(const StageTerms& st, int j) { return st.dc ? st.dc->cEl[j] : st.cEl[j]; }
__device__ __forceinline__ double gamma_of(const StageTerms& st) { return st.dc ? st.dc->gamma : st.gamma; }
__device__ __forceinline__ double qgamma_of(const StageTerms& st) { return st.dc ? st.dc->qgamma : st.qgamma; }
__device__ __forceinline__ float cIh_of(const StageTerms& st, int j) { return st.dc ? st.dc->cIh[j] : st.cIh[j]; }
__device__ __forceinline__ float cIl_of(const StageTerms& st, int j) { return st.dc ? st.dc->cIl[j] : st.cIl[j]; }
__device__ __forceinline__ float gh_of(const StageTerms& st) { return st.dc ? st.dc->gh : st.gh; }
__device__ __forceinline__ float gl_of(const StageTerms& st) { return st.dc ? st.dc->gl : st.gl; }
__device__ __forceinline__ float qgh_of(const StageTerms& st) { return st.dc ? st.dc->qgh : st.qgh; }
__device__ __forceinline__ float qgl_of(const StageTerms& st) { return st.dc ? st.dc->qgl : st.qgl; }
// batch members that reached t_final (or failed) skip all work
#define PF_SKIP_INACTIVE(g) \
    if ((g).active && *(g).active == 0) return
// a batch member's state alternates between its two state buffers (an
// accepted attempt flips the parity instead of copying y_new over y)
__device__ __forceinline__ bool y_swapped(const Geo& g) { return g.ypar && *g.ypar; }

template <typename T2>
__device__ __forceinline__ double2 load_f(const void* p, long long i) {
    return to_d2(reinterpret_cast<const T2*>(p)[i]);
}

// r += c * v (complex v, real c), FP64
__device__ __forceinline__ void axpy(double2& r, double c, double2 v) {
    r.x = fma(c, v.x, r.x);
    r.y = fma(c, v.y, r.y);
}

// Exact float -> double by bit manipulation (FP32 subnormals flush to zero),
// keeping the conversion off the FP64 pipe.
__device__ __forceinline__ double f2d_bits(float x) {
    const unsigned u = __float_as_uint(x);
    const unsigned ex = (u >> 23) & 0xffu, sign = u & 0x80000000u, man = u & 0x7fffffu;
    if (ex == 0u) return __hiloint2double((int)sign, 0);
    unsigned hi;
    if (ex == 0xffu)
        hi = sign | 0x7ff00000u | (man >> 3) | (man ? 0x80000u : 0u);
    else
        hi = sign | ((ex + 896u) << 20) | (man >> 3);
    return __hiloint2double((int)hi, (int)(man << 29));
}

// double -> float, round to nearest even, by bit manipulation (results below
// the FP32 normal range flush to zero).
__device__ __forceinline__ float d2f_bits(double d) {
    const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
    const unsigned sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu);
    if (e == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (((hi & 0xfffffu) | lo) ? 0x400000u : 0u));
    int fe = e - 896;
    if (fe <= 0) return __uint_as_float(sign);
    unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned rem = lo & 0x1fffffffu, half = 0x10000000u;
    if (rem > half || (rem == half && (m & 1u))) {
        m += 1u;
        if (m == 0x800000u) {
            m = 0u;
            ++fe;
        }
    }
    if (fe >= 255) return __uint_as_float(sign | 0x7f800000u);
    return __uint_as_float(sign | ((unsigned)fe << 23) | m);
}

// Double-single accumulation (hi, lo) += (ch + cl) * f for an FP32 value f:
// the product ch*f is split exactly with an FMA, cl*f is added to its error,
// and the sum uses the two-sum error-free transformation (no contraction:
// explicitly rounded intrinsics).  Carries ~48 bits, so FP32 stage terms enter
// the FP64 combination without passing through the narrow FP64 pipe.
__device__ __forceinline__ void ds_add_prod(float& sh, float& sl, float ch, float cl, float f) {
    const float p = __fmul_rn(ch, f);
    float e = __fmaf_rn(ch, f, -p);
    e = __fmaf_rn(cl, f, e);
    const float s = __fadd_rn(sh, p);
    const float bb = __fsub_rn(s, sh);
    const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(err, e));
}

struct DS2 {
    float xh = 0.f, xl = 0.f, yh = 0.f, yl = 0.f;
    __device__ __forceinline__ void add(float ch, float cl, float2 f) {
        ds_add_prod(xh, xl, ch, cl, f.x);
        ds_add_prod(yh, yl, ch, cl, f.y);
    }
    __device__ __forceinline__ void flush(double2& r) const {
        r.x += f2d_bits(xh) + f2d_bits(xl);
        r.y += f2d_bits(yh) + f2d_bits(yl);
    }
};

// ---------------------------------------------------------------------------
// Double-float numbers h + l (two FP32 words, |l| <= ulp(h)/2, ~46 significant
// bits).  The FP32-bulk stage combination keeps the stage vectors z_j, lambda,
// the implicit factor q and every running sum in this form, so that it runs on
// the FP32 pipe at close to FP64 accuracy (error-free transformations: Dekker
// and Knuth two-sum / two-product with an FMA, explicitly rounded intrinsics so
// that no contraction changes them).
// ---------------------------------------------------------------------------
struct DF {
    float h, l;
};

// (h, e) = two_sum(a, b): h = fl(a + b), a + b = h + e exactly
__device__ __forceinline__ DF df_two_sum(float a, float b) {
    const float h = __fadd_rn(a, b);
    const float bb = __fsub_rn(h, a);
    return DF{h, __fadd_rn(__fsub_rn(a, __fsub_rn(h, bb)), __fsub_rn(b, bb))};
}

// FP32 value of an FP64 one, given as its two 32-bit words, truncated to 24
// significant bits (below the FP32 normal range: signed zero; above it:
// infinity; NaN stays NaN).  In range the exponent field is rebiased in place
// and one funnel shift brings exponent and leading mantissa bits together.
__device__ __forceinline__ float f32_trunc_hilo(unsigned hi, unsigned lo) {
    const unsigned sign = hi & 0x80000000u;
    const unsigned ef = (hi >> 20) & 0x7ffu;  // FP64 biased exponent; FP32 normal range: 897..1150
    unsigned r = __funnelshift_l(lo, hi - (896u << 20), 3) | sign;
    if (ef - 897u >= 254u)
        r = ef <= 896u ? sign
                       : sign | 0x7f800000u | (ef == 2047u && ((hi & 0xfffffu) | lo) != 0u ? 0x400000u : 0u);
    return __uint_as_float(r);
}
__device__ __forceinline__ float f32_trunc_bits(double d) {
    return f32_trunc_hilo((unsigned)__double2hiint(d), (unsigned)__double2loint(d));
}

// FP64 -> double-float: h = d truncated to 24 significant bits (exact in both
// types), l = d - h (one exact FP64 subtraction) truncated to FP32; h + l
// carries at least 47 significant bits.  Bit operations only, apart from the
// subtraction.  Double-float -> FP64: one FP64 addition.
__device__ __forceinline__ DF df_from_d(double d) {
    const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
    const bool normal = ((hi >> 20) & 0x7ffu) > 896u;  // |d| at or above the FP32 normal range
    const unsigned lh = lo & 0xe0000000u;
    const double hd = normal ? __hiloint2double((int)hi, (int)lh) : 0.0;
    return DF{normal ? f32_trunc_hilo(hi, lh) : 0.0f, f32_trunc_bits(d - hd)};
}
__device__ __forceinline__ double df_to_d(DF a) { return f2d_bits(a.h) + f2d_bits(a.l); }

__device__ __forceinline__ DF df_add(DF a, DF b) {
    const DF s = df_two_sum(a.h, b.h);
    return df_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}

__device__ __forceinline__ DF df_mul(DF a, DF b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return df_two_sum(p, e);
}

// 1 / a: FP32 reciprocal, one Newton step carried in double-float
// (1 - a.h r is exact for r = fl(1 / a.h))
__device__ __forceinline__ DF df_rcp(DF a) {
    const float r = __frcp_rn(a.h);
    float t = __fmaf_rn(-a.h, r, 1.0f);
    t = __fmaf_rn(-a.l, r, t);
    return df_two_sum(r, __fmul_rn(r, t));
}

// running sum (sh, sl) += (ch + cl) (zh + zl), the cl zl term dropped; the sum
// is normalised once at the end (df_two_sum(sh, sl))
__device__ __forceinline__ void df_acc(float& sh, float& sl, float ch, float cl, float zh, float zl) {
    const float p = __fmul_rn(ch, zh);
    float e = __fmaf_rn(ch, zh, -p);
    e = __fmaf_rn(ch, zl, e);
    e = __fmaf_rn(cl, zh, e);
    const DF s = df_two_sum(sh, p);
    sh = s.h;
    sl = __fadd_rn(sl, __fadd_rn(s.l, e));
}

// complex running sums sum_j c_j z_j of the FP32-bulk combination
struct DFAcc {
    float xh = 0.f, xl = 0.f, yh = 0.f, yl = 0.f;
    __device__ __forceinline__ void add(float ch, float cl, DF zx, DF zy) {
        df_acc(xh, xl, ch, cl, zx.h, zx.l);
        df_acc(yh, yl, ch, cl, zy.h, zy.l);
    }
    __device__ __forceinline__ void add(float ch, float cl, float2 f) {
        ds_add_prod(xh, xl, ch, cl, f.x);
        ds_add_prod(yh, yl, ch, cl, f.y);
    }
    __device__ __forceinline__ DF x() const { return df_two_sum(xh, xl); }
    __device__ __forceinline__ DF y() const { return df_two_sum(yh, yl); }
};

__device__ __forceinline__ double lam_at(const Geo& g, const Phys& ph, int f, long long gi, double kx, double ky,
                                         double kz) {
    return g.lam ? g.lam[gi] : lambda_k(ph, f, kx, ky, kz);
}

// Model constants in the compute type, converted once per thread (a
// per-element double->float conversion would run on the narrow FP64 pipe).
// the model constants in the compute type (rounded on the host)
template <typename T>
__device__ __forceinline__ const PhysT<T>& phys_t(const Phys& ph);
template <>
__device__ __forceinline__ const PhysT<double>& phys_t<double>(const Phys& ph) { return ph.t64; }
template <>
__device__ __forceinline__ const PhysT<float>& phys_t<float>(const Phys& ph) { return ph.t32; }

// wave number of axis a (0 = x half spectrum, 1 = y, 2 = z) in the compute type
template <typename T>
__device__ __forceinline__ T kval(const Geo& g, int a, int i);
template <>
__device__ __forceinline__ double kval<double>(const Geo& g, int a, int i) {
    return a == 0 ? g.kx[i] : (a == 1 ? g.ky[i] : g.kz[i]);
}
template <>
__device__ __forceinline__ float kval<float>(const Geo& g, int a, int i) {
    return a == 0 ? g.kx32[i] : (a == 1 ? g.ky32[i] : g.kz32[i]);
}

template <typename T2>
__device__ __forceinline__ T2 narrow(double2 a);
template <>
__device__ __forceinline__ double2 narrow<double2>(double2 a) { return a; }
template <>
__device__ __forceinline__ float2 narrow<float2>(double2 a) { return make_float2(d2f_bits(a.x), d2f_bits(a.y)); }

template <typename T>
static int strided_tile(int n, int nbuf, int budget) {
    int tx = 16;
    while (tx > 1 && (size_t)nbuf * tx * n * sizeof(typename Cx<T>::t) > (size_t)budget) tx >>= 1;
    return tx;
}

template <typename T>
static int tile_cols(const Geo& g, int n, int nbuf, int budget) {
    int tx = strided_tile<T>(n, nbuf, budget);
    // no wider than the (odd) half-spectrum row
    while (tx > 1 && tx / 2 >= g.nxh) tx >>= 1;
    return tx;
}

// tuned width (0 = untuned) capped by what fits the shared-memory budget
template <typename T>
static int tuned_cols(const Geo& g, int tuned, int n, int nbuf, int budget) {
    if (tuned <= 0) return tile_cols<T>(g, n, nbuf, nbuf == 4 ? 64 * 1024 : 96 * 1024);
    const int cap = tile_cols<T>(g, n, nbuf, budget);
    int tx = 1;
    while (tx * 2 <= tuned && tx * 2 <= 16) tx *= 2;
    return tx < cap ? tx : cap;
}

template <typename K>
static void set_smem(K kern, size_t bytes) {
    if (bytes > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// compile-time radix-16 support dispatch (R16C), from the axis plan
#define PF_R16_SWITCH(flag, ...)       \
    if (flag) {                        \
        constexpr bool R16C = true;    \
        __VA_ARGS__;                   \
    } else {                           \
        constexpr bool R16C = false;   \
        __VA_ARGS__;                   \
    }

// asynchronous global -> shared copy of BYTES (4, 8 or 16) bytes; the data
// never passes through registers, so a thread can have any number in flight
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(gmem), "n"(BYTES));
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Launch dispatch of a column pass over the tile width (TXC), the radix-16
// flag (R16C) and the compiled plan (PIDC): FP32 kernels with tile widths 8
// or 16 run the compile-time plan when the axis plan is one of the compiled
// ones, everything else the generic stages.
#define PF_PID_CASE(K_, tx, ...)            \
    case K_: {                              \
        constexpr int PIDC = K_;            \
        constexpr bool R16C = false;        \
        if ((tx) == 16) {                   \
            constexpr int TXC = 16;         \
            __VA_ARGS__;                    \
        } else {                            \
            constexpr int TXC = 8;          \
            __VA_ARGS__;                    \
        }                                   \
    } break;
#define PF_COL_SWITCH(T_, plan, tx, ...)                                                          \
    do {                                                                                          \
        int pid_ = 0;                                                                             \
        if (sizeof(T_) == 4 && ((tx) == 8 || (tx) == 16)) pid_ = fixed_plan_id(plan);              \
        if constexpr (sizeof(T_) == 4) {                                                          \
            switch (pid_) {                                                                       \
                PF_PID_CASE(1, tx, __VA_ARGS__)                                                   \
                PF_PID_CASE(2, tx, __VA_ARGS__)                                                   \
                PF_PID_CASE(3, tx, __VA_ARGS__)                                                   \
                PF_PID_CASE(4, tx, __VA_ARGS__)                                                   \
                PF_PID_CASE(5, tx, __VA_ARGS__)                                                   \
                PF_PID_CASE(6, tx, __VA_ARGS__)                                                   \
                PF_PID_CASE(7, tx, __VA_ARGS__)                                                   \
                PF_PID_CASE(8, tx, __VA_ARGS__)                                                   \
                PF_PID_CASE(9, tx, __VA_ARGS__)                                                   \
                PF_PID_CASE(10, tx, __VA_ARGS__)                                                  \
                PF_PID_CASE(11, tx, __VA_ARGS__)                                                  \
                default: break;                                                                   \
            }                                                                                     \
        }                                                                                         \
        if (pid_ == 0) {                                                                          \
            constexpr int PIDC = 0;                                                               \
            PF_R16_SWITCH((plan).has16, PF_TX_SWITCH(tx, __VA_ARGS__));                            \
        }                                                                                         \
    } while (0)

// as PF_COL_SWITCH, with compiled plans for tile width 8 only (passes whose
// wider tiles do not fit shared memory)
#define PF_PID_CASE8(K_, ...)               \
    case K_: {                              \
        constexpr int PIDC = K_;            \
        constexpr bool R16C = false;        \
        constexpr int TXC = 8;              \
        __VA_ARGS__;                        \
    } break;
#define PF_COL_SWITCH8(T_, plan, tx, ...)                                                         \
    do {                                                                                          \
        int pid_ = 0;                                                                             \
        if (sizeof(T_) == 4 && (tx) == 8) pid_ = fixed_plan_id(plan);                             \
        if constexpr (sizeof(T_) == 4) {                                                          \
            switch (pid_) {                                                                       \
                PF_PID_CASE8(1, __VA_ARGS__)                                                      \
                PF_PID_CASE8(2, __VA_ARGS__)                                                      \
                PF_PID_CASE8(3, __VA_ARGS__)                                                      \
                PF_PID_CASE8(4, __VA_ARGS__)                                                      \
                PF_PID_CASE8(5, __VA_ARGS__)                                                      \
                PF_PID_CASE8(6, __VA_ARGS__)                                                      \
                PF_PID_CASE8(7, __VA_ARGS__)                                                      \
                PF_PID_CASE8(8, __VA_ARGS__)                                                      \
                PF_PID_CASE8(9, __VA_ARGS__)                                                      \
                PF_PID_CASE8(10, __VA_ARGS__)                                                     \
                PF_PID_CASE8(11, __VA_ARGS__)                                                     \
                default: break;                                                                   \
            }                                                                                     \
        }                                                                                         \
        if (pid_ == 0) {                                                                          \
            constexpr int PIDC = 0;                                                               \
            PF_R16_SWITCH((plan).has16, PF_TX_SWITCH(tx, __VA_ARGS__));                            \
        }                                                                                         \
    } while (0)

// compile-time tile width dispatch
#define PF_TX_SWITCH(tx, ...)                 \
    switch (tx) {                             \
        case 16: {                            \
            constexpr int TXC = 16;           \
            __VA_ARGS__;                      \
        } break;                              \
        case 8: {                             \
            constexpr int TXC = 8;            \
            __VA_ARGS__;                      \
        } break;                              \
        case 4: {                             \
            constexpr int TXC = 4;            \
            __VA_ARGS__;                      \
        } break;                              \
        case 2: {                             \
            constexpr int TXC = 2;            \
            __VA_ARGS__;                      \
        } break;                              \
        default: {                            \
            constexpr int TXC = 1;            \
            __VA_ARGS__;                      \
        } break;                              \
    }

// ---------------------------------------------------------------------------
// FP32-bulk stage combination in double-float (one element gi):
//   r = y + lambda sum_j (dt A^I_ij) z_j + sum_j (dt A^E_ij) f^E_j,  z_i = q r
// z_j are float4 {Re h, Im h, Re l, Im l} (or y itself where st.mY says so),
// lambda and q are float2 {h, l}; y enters through one FP64 split per
// component.  Writes z_i and (first stage of a step) the q table; returns
// fl32(z_i) for the transform.
// ---------------------------------------------------------------------------
__device__ __forceinline__ DF df_one_minus(DF c, DF lam) { return df_add(DF{1.f, 0.f}, df_mul(DF{-c.h, -c.l}, lam)); }

// where the stage coefficients of a FP32-bulk combination live: DC = 0 in the
// kernel parameters (direct operands, no loads), DC = 1 behind st.dc (device
// copies written by the batch round kernels), DC = -1 decided per call
template <int DC>
struct CoefSrc {
    const StageTerms& st;
    __device__ __forceinline__ bool dev() const { return DC < 0 ? st.dc != nullptr : DC > 0; }
    __device__ __forceinline__ float Ih(int j) const { return dev() ? st.dc->cIh[j] : st.cIh[j]; }
    __device__ __forceinline__ float Il(int j) const { return dev() ? st.dc->cIl[j] : st.cIl[j]; }
    __device__ __forceinline__ float Eh(int j) const { return dev() ? st.dc->cEh[j] : st.cEh[j]; }
    __device__ __forceinline__ float El(int j) const { return dev() ? st.dc->cEl[j] : st.cEl[j]; }
    __device__ __forceinline__ DF gamma() const { return dev() ? DF{st.dc->gh, st.dc->gl} : DF{st.gh, st.gl}; }
    __device__ __forceinline__ DF qgamma() const { return dev() ? DF{st.dc->qgh, st.dc->qgl} : DF{st.qgh, st.qgl}; }
};

// row of the double-float lambda and q tables for element gi = f NK + k:
// gi itself, or with shared phi rows (g.lam2) k for X and NK + k for any phi
__device__ __forceinline__ long long lam_row(const Geo& g, long long gi) {
    return (g.lam2 && gi >= g.NK) ? g.NK + gi % g.NK : gi;
}

// at most MAXT earlier-stage terms (compile-time bound: fewer registers);
// Idx: element index type (unsigned where 4 NK < 2^32: one-instruction
// address arithmetic); ti: the element's row of the lambda and q tables
// (lam_row)
template <int MAXT = kMaxStages, int DC = -1, typename Idx = long long>
__device__ __forceinline__ float2 stage_value_df(const Geo& g, const StageTerms& st, const double2* __restrict__ y,
                                                 Idx gi, Idx ti, float4* __restrict__ zout) {
    const CoefSrc<DC> cs{st};
    // every load first (independent, all in flight together), then the sums
    const bool need_lam = st.mI != 0u || st.qout || st.has_gamma;
    const bool load_q = st.has_gamma && st.qin;
    const double2 yv = __ldg(y + gi);
    const float2 lt = need_lam ? __ldg(g.lamdf + ti) : make_float2(0.f, 0.f);
    const float2 qt = load_q ? __ldg(reinterpret_cast<const float2*>(st.qin) + ti) : make_float2(1.f, 0.f);
    const unsigned mz = st.mI & ~st.mY;
    float4 zv[MAXT > 0 ? MAXT : 1];
    float2 fv[MAXT > 0 ? MAXT : 1];
#pragma unroll
    for (int j = 0; j < MAXT; ++j) {
        zv[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        fv[j] = make_float2(0.f, 0.f);
        if (j < st.n) {
            if ((mz >> j) & 1u) zv[j] = __ldg(reinterpret_cast<const float4*>(st.z[j]) + gi);
            if ((st.mE >> j) & 1u) fv[j] = __ldg(reinterpret_cast<const float2*>(st.f[j]) + gi);
        }
    }
    const DF yx = df_from_d(yv.x), yy = df_from_d(yv.y);
    DFAcc I, E;
#pragma unroll
    for (int j = 0; j < MAXT; ++j) {
        if (j < st.n) {
            if ((st.mI >> j) & 1u) {
                const float ch = cs.Ih(j), cl = cs.Il(j);
                if ((st.mY >> j) & 1u)
                    I.add(ch, cl, yx, yy);
                else
                    I.add(ch, cl, DF{zv[j].x, zv[j].z}, DF{zv[j].y, zv[j].w});
            }
            if ((st.mE >> j) & 1u) E.add(cs.Eh(j), cs.El(j), fv[j]);
        }
    }
    DF rx = df_add(yx, E.x()), ry = df_add(yy, E.y());
    if (need_lam) {
        const DF lam{lt.x, lt.y};
        if (st.mI != 0u) {
            rx = df_add(rx, df_mul(lam, I.x()));
            ry = df_add(ry, df_mul(lam, I.y()));
        }
        // (with shared phi rows the three phi fields would write the same row)
        if (st.qout && (!g.lam2 || (long long)gi < 2 * g.NK)) {
            const DF q = df_rcp(df_one_minus(cs.qgamma(), lam));
            reinterpret_cast<float2*>(st.qout)[ti] = make_float2(q.h, q.l);
        }
        if (st.has_gamma) {
            const DF q = load_q ? DF{qt.x, qt.y} : df_rcp(df_one_minus(cs.gamma(), lam));
            rx = df_mul(rx, q);
            ry = df_mul(ry, q);
        }
    }
    if (zout) zout[gi] = make_float4(rx.h, ry.h, rx.l, ry.l);
    return make_float2(rx.h, ry.h);
}

// FP32-bulk step completion (double-float):
//   y_n = y + [lambda sum_j (dt b^I_j) z_j + sum_j (dt b^E_j) f^E_j]
// with the bracket rounded to FP64 once and added to the FP64 state; returns
// the local error estimate (the same sums with dt (b - bt)) in FP32.  MAXT,
// DC and Idx as in stage_value_df.
template <int MAXT = kMaxStages, int DC = -1, typename Idx = long long>
__device__ __forceinline__ float2 final_value_df(const Geo& g, const StageTerms& bt, const StageTerms& dt,
                                                 int want_lte, const double2* __restrict__ y, Idx gi, Idx ti,
                                                 double2* __restrict__ ynew) {
    const CoefSrc<DC> cb{bt}, cd{dt};
    const unsigned lmI = want_lte ? dt.mI : 0u, lmE = want_lte ? dt.mE : 0u;
    const unsigned mI = bt.mI | lmI, mE = bt.mE | lmE, mz = mI & ~bt.mY;
    // every load first, then the sums
    const double2 yv = __ldg(y + gi);
    const float2 lt = mI != 0u ? __ldg(g.lamdf + ti) : make_float2(0.f, 0.f);
    float4 zv[MAXT];
    float2 fv[MAXT];
#pragma unroll
    for (int j = 0; j < MAXT; ++j) {
        zv[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        fv[j] = make_float2(0.f, 0.f);
        if (j < bt.n) {
            if ((mz >> j) & 1u) zv[j] = __ldg(reinterpret_cast<const float4*>(bt.z[j]) + gi);
            if ((mE >> j) & 1u) fv[j] = __ldg(reinterpret_cast<const float2*>(bt.f[j]) + gi);
        }
    }
    DF yx{0.f, 0.f}, yy{0.f, 0.f};
    if ((bt.mY & mI) != 0u) {
        yx = df_from_d(yv.x);
        yy = df_from_d(yv.y);
    }
    // y_n in double-float; the local error estimate (an estimate, transformed
    // and normed in FP32 next) in plain FP32 from the leading words
    DFAcc Ib, Eb;
    float dIx = 0.f, dIy = 0.f, dEx = 0.f, dEy = 0.f;
#pragma unroll
    for (int j = 0; j < MAXT; ++j) {
        if (j < bt.n) {
            const bool bI = (bt.mI >> j) & 1u, bE = (bt.mE >> j) & 1u;
            const bool lI = (lmI >> j) & 1u, lE = (lmE >> j) & 1u;
            if (bI || lI) {
                DF zx = yx, zy = yy;
                if (!((bt.mY >> j) & 1u)) {
                    zx = DF{zv[j].x, zv[j].z};
                    zy = DF{zv[j].y, zv[j].w};
                }
                if (bI) Ib.add(cb.Ih(j), cb.Il(j), zx, zy);
                if (lI) {
                    dIx = __fmaf_rn(cd.Ih(j), zx.h, dIx);
                    dIy = __fmaf_rn(cd.Ih(j), zy.h, dIy);
                }
            }
            if (bE) Eb.add(cb.Eh(j), cb.El(j), fv[j]);
            if (lE) {
                dEx = __fmaf_rn(cd.Eh(j), fv[j].x, dEx);
                dEy = __fmaf_rn(cd.Eh(j), fv[j].y, dEy);
            }
        }
    }
    const DF lam{lt.x, lt.y};
    const DF dx = df_add(df_mul(lam, Ib.x()), Eb.x()), dy = df_add(df_mul(lam, Ib.y()), Eb.y());
    ynew[gi] = make_double2(yv.x + df_to_d(dx), yv.y + df_to_d(dy));
    return make_float2(__fmaf_rn(lam.h, dIx, dEx), __fmaf_rn(lam.h, dIy, dEy));
}

// ---------------------------------------------------------------------------
// z pass: elastic Green's contraction (homogeneous cubic modulus)
//   e^_v(k) = sum_q B_vq(n) h^_q(k) / N,  n = k/|k|, B(0) = 0
//   B_vq(n) = eps*_v:C:eps*_q - (sigma*_v n) . Omega(n) . (sigma*_q n),
//   Omega^{-1}_ik = C44 d_ik + (C12 + C44) n_i n_k + (C11 - C12 - 2 C44) d_ik n_i^2
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void elastic_kernel(const PhysT<T>& pt, T kx, T ky, T kz, T Bm[3][3]) {
    const T k2 = kx * kx + ky * ky + kz * kz;
    if (k2 == (T)0) {
#pragma unroll
        for (int v = 0; v < 3; ++v)
#pragma unroll
            for (int q = 0; q < 3; ++q) Bm[v][q] = (T)0;
        return;
    }
    const T inv = (T)1 / sqrt(k2);
    const T n0 = kx * inv, n1 = ky * inv, n2 = kz * inv;
    const T C44 = pt.C44, Cm = pt.Cm, Ca = pt.Ca;
    const T a = C44 + Cm * n0 * n0 + Ca * n0 * n0;
    const T b = C44 + Cm * n1 * n1 + Ca * n1 * n1;
    const T c = C44 + Cm * n2 * n2 + Ca * n2 * n2;
    const T d = Cm * n0 * n1, e = Cm * n0 * n2, f = Cm * n1 * n2;
    // inverse of the symmetric acoustic tensor by cofactors
    const T A11 = b * c - f * f, A12 = e * f - d * c, A13 = d * f - b * e;
    const T A22 = a * c - e * e, A23 = d * e - a * f, A33 = a * b - d * d;
    const T idet = (T)1 / (a * A11 + d * A12 + e * A13);
    T s[3][3];
#pragma unroll
    for (int v = 0; v < 3; ++v) {
        const T* S = pt.sig[v];  // xx yy zz yz xz xy
        s[v][0] = S[0] * n0 + S[5] * n1 + S[4] * n2;
        s[v][1] = S[5] * n0 + S[1] * n1 + S[3] * n2;
        s[v][2] = S[4] * n0 + S[3] * n1 + S[2] * n2;
    }
    T Os[3][3];  // Omega s_q
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        Os[q][0] = (A11 * s[q][0] + A12 * s[q][1] + A13 * s[q][2]) * idet;
        Os[q][1] = (A12 * s[q][0] + A22 * s[q][1] + A23 * s[q][2]) * idet;
        Os[q][2] = (A13 * s[q][0] + A23 * s[q][1] + A33 * s[q][2]) * idet;
    }
#pragma unroll
    for (int v = 0; v < 3; ++v)
#pragma unroll
        for (int q = 0; q < 3; ++q)
            Bm[v][q] = pt.cvq[v][q] - (s[v][0] * Os[q][0] + s[v][1] * Os[q][1] + s[v][2] * Os[q][2]);
}

}  // namespace pf
