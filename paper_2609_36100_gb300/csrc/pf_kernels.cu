// Pass kernels of the pseudospectral ImEx-ARK right-hand side (Sec. 4.2/4.4
// of the paper) on sm_103a.
//
// One explicit right-hand-side evaluation f^E(z) is nine memory passes over
// field-major arrays ([field][z][y][x] real, [field][kz][ky][kx] half
// spectrum), each one shared-memory FFT along one axis with the pointwise
// work of that point of the method fused into it:
//   z: stage assembly + diagonal implicit solve (Eq. ARK_stage) + inverse FFT
//   y: inverse FFT
//   x: C2R -> real X, phi_v; h(phi_v) -> R2C (or the whole RHS when the
//      eigenstrains vanish)
//   y: forward FFT of h          z: forward FFT, Green's contraction
//   y: inverse FFT of e          B_vq(k/|k|) h^_q, inverse FFT
//   x: C2R of e, KKS mu, g_v, q -> R2C        y: forward FFT
//   z: forward FFT + k-space scaling -> f^E (-M k^2, -L)
// Step completion (Eq. ARK_method), the embedded local error (Eq.
// ARK_embedding) and its WRMS norm (Eqs. wrms_norm, wrms_weights) are three
// more passes.  Template parameter T is the compute type of the transforms
// and RHS (double, or float for the FP32-bulk form); the state and stage
// vectors are always FP64.
#include <cstdio>

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
// batch members that reached t_final (or failed) skip all work
#define PF_SKIP_INACTIVE(g) \
    if ((g).active && *(g).active == 0) return

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

__device__ __forceinline__ double lam_at(const Geo& g, const Phys& ph, int f, long long gi, double kx, double ky,
                                         double kz) {
    return g.lam ? g.lam[gi] : lambda_k(ph, f, kx, ky, kz);
}

// Model constants in the compute type, converted once per thread (a
// per-element double->float conversion would run on the narrow FP64 pipe).
template <typename T>
struct PhysT {
    T Bv, Bm, inv2Av, inv2Am, A0m, A0v, Am, Av, wb2, ie, twoAm;
    T w[3][3];
    T C44, Cm, Ca;
    T sig[3][6];
    T cvq[3][3];
    __device__ __forceinline__ explicit PhysT(const Phys& ph) {
        Bv = (T)ph.Bv;
        Bm = (T)ph.Bm;
        inv2Av = (T)ph.inv2Av;
        inv2Am = (T)ph.inv2Am;
        A0m = (T)ph.A0m;
        A0v = (T)ph.A0v;
        Am = (T)ph.Am;
        Av = (T)ph.Av;
        wb2 = (T)(2.0 * ph.wbar);
        ie = (T)(1.0 / ph.pair_eps);
        twoAm = (T)(2.0 * ph.Am);
        C44 = (T)ph.C44;
        Cm = (T)ph.Cmix;
        Ca = (T)ph.Caniso;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                w[a][b] = (T)ph.w[a][b];
                cvq[a][b] = (T)ph.cvq[a][b];
            }
#pragma unroll
            for (int b = 0; b < 6; ++b) sig[a][b] = (T)ph.sig[a][b];
        }
    }
};

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
// z pass: stage assembly + implicit solve + inverse FFT along z
//   r = y + sum_j (dt A^I_ij) lambda z_j + (dt A^E_ij) f^E_j
//   z_i = r / (1 - dt A^I_ii lambda)
// The assembly is the first FFT stage's load: each element is formed once.
// ---------------------------------------------------------------------------
template <typename T, int TX>
__global__ void __launch_bounds__(kThreads) k_z_stage(Geo g, Phys ph, const double2* __restrict__ y, StageTerms st,
                                                      double2* __restrict__ zout,
                                                      typename Cx<T>::t* __restrict__ W) {
    PF_SKIP_INACTIVE(g);
    using T2 = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smraw[];
    T2* A = reinterpret_cast<T2*>(smraw);
    T2* B = A + TX * g.nz;
    const int f = blockIdx.z, ky = blockIdx.y, kx0 = blockIdx.x * TX;
    const int ncol = min(TX, g.nxh - kx0);
    const long long base = (long long)f * g.NK + (long long)ky * g.nxh + kx0;
    const long long zs = (long long)g.ny * g.nxh;
    const double kyv = g.ky[ky];
    auto src = [&](int kz, int col) -> T2 {
        if (col >= ncol) return T2{0, 0};
        const long long gi = base + kz * zs + col;
        double2 r = y[gi];
        const double lam = lam_at(g, ph, f, gi, g.kx[kx0 + col], kyv, g.kz[kz]);
        DS2 fs;
        double2 zi = make_double2(0.0, 0.0);  // sum_j (dt A^I_ij) z_j, times lambda below
#pragma unroll
        for (int j = 0; j < kMaxStages; ++j) {
            if (j < st.n) {
                if ((st.mI >> j) & 1u) axpy(zi, cI_of(st, j), st.z[j][gi]);
                if ((st.mE >> j) & 1u) {
                    if (sizeof(T) == 4)
                        fs.add(cEh_of(st, j), cEl_of(st, j), reinterpret_cast<const float2*>(st.f[j])[gi]);
                    else
                        axpy(r, cE_of(st, j), load_f<T2>(st.f[j], gi));
                }
            }
        }
        axpy(r, lam, zi);
        if (sizeof(T) == 4) fs.flush(r);
        if (st.qout) st.qout[gi] = 1.0 / (1.0 - qgamma_of(st) * lam);
        if (st.has_gamma) {
            const double q = st.qin ? st.qin[gi] : 1.0 / (1.0 - gamma_of(st) * lam);
            r.x *= q;
            r.y *= q;
        }
        if (zout) zout[gi] = r;
        return narrow<T2>(r);
    };
    auto dst = [&](int kz, int col, T2 v) {
        if (col < ncol) W[base + kz * zs + col] = v;
    };
    fft_cols<+1, TX>(g.pz, A, B, src, dst);
}

template <typename T>
void launch_z_stage(const Geo& g, const Phys& ph, const double2* y, const StageTerms& st, double2* zout, void* W,
                    cudaStream_t s) {
    using T2 = typename Cx<T>::t;
    const int TX = tuned_cols<T>(g, g.tx_z, g.nz, 2, 128 * 1024);
    const size_t sm = 2 * (size_t)TX * g.nz * sizeof(T2);
    dim3 grid((g.nxh + TX - 1) / TX, g.ny, 4);
    PF_TX_SWITCH(TX, set_smem(k_z_stage<T, TXC>, sm);
                 k_z_stage<T, TXC><<<grid, kThreads, sm, s>>>(g, ph, y, st, zout, reinterpret_cast<T2*>(W)))
}

// ---------------------------------------------------------------------------
// y pass: in-place complex FFT along y of nf fields
// ---------------------------------------------------------------------------
template <typename T, int SIGN, int TX>
__global__ void __launch_bounds__(kThreads) k_y_pass(Geo g, typename Cx<T>::t* __restrict__ buf) {
    PF_SKIP_INACTIVE(g);
    using T2 = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smraw[];
    T2* A = reinterpret_cast<T2*>(smraw);
    T2* B = A + TX * g.ny;
    const int f = blockIdx.z, kz = blockIdx.y, kx0 = blockIdx.x * TX;
    const int ncol = min(TX, g.nxh - kx0);
    T2* base = buf + (long long)f * g.NK + (long long)kz * g.ny * g.nxh + kx0;
    const int ys = g.nxh;
    auto src = [&](int ky, int col) -> T2 { return col < ncol ? base[ky * ys + col] : T2{0, 0}; };
    auto dst = [&](int ky, int col, T2 v) {
        if (col < ncol) base[ky * ys + col] = v;
    };
    fft_cols<SIGN, TX, true>(g.py, A, B, src, dst);
}

template <typename T>
void launch_y_pass(const Geo& g, void* buf, int nf, int sign, cudaStream_t s) {
    using T2 = typename Cx<T>::t;
    const int TX = tuned_cols<T>(g, g.tx_y, g.ny, 2, 128 * 1024);
    const size_t sm = 2 * (size_t)TX * g.ny * sizeof(T2);
    dim3 grid((g.nxh + TX - 1) / TX, g.nz, nf);
    if (sign > 0) {
        PF_TX_SWITCH(TX, set_smem(k_y_pass<T, 1, TXC>, sm);
                     k_y_pass<T, 1, TXC><<<grid, kThreads, sm, s>>>(g, reinterpret_cast<T2*>(buf)))
    } else {
        PF_TX_SWITCH(TX, set_smem(k_y_pass<T, -1, TXC>, sm);
                     k_y_pass<T, -1, TXC><<<grid, kThreads, sm, s>>>(g, reinterpret_cast<T2*>(buf)))
    }
}

// ---------------------------------------------------------------------------
// z pass, forward: FFT along z then k-space scaling (the last stage's store)
//   mode 0: y^ = W / N  -> FP64                                  (set_state)
//   mode 1: f^E_X = -M k^2 q^/N, f^E_phi = -L g^/N -> compute type (stages)
//   mode 2: same scaling -> FP64                                  (ABI f^E)
// ---------------------------------------------------------------------------
template <typename T, typename OT2, int TX>
__global__ void __launch_bounds__(kThreads) k_z_fwd(Geo g, Phys ph, const typename Cx<T>::t* __restrict__ W,
                                                    OT2* __restrict__ out, int mode) {
    PF_SKIP_INACTIVE(g);
    using T2 = typename Cx<T>::t;
    using OT = decltype(OT2{}.x);
    extern __shared__ __align__(16) unsigned char smraw[];
    T2* A = reinterpret_cast<T2*>(smraw);
    T2* B = A + TX * g.nz;
    const int f = blockIdx.z, ky = blockIdx.y, kx0 = blockIdx.x * TX;
    const int ncol = min(TX, g.nxh - kx0);
    const long long base = (long long)f * g.NK + (long long)ky * g.nxh + kx0;
    const long long zs = (long long)g.ny * g.nxh;
    const double invN = 1.0 / (double)g.N;
    const T mN = (T)(-ph.M * invN), lN = (T)(-ph.L * invN);
    const T kyv = kval<T>(g, 1, ky);
    auto src = [&](int kz, int col) -> T2 { return col < ncol ? W[base + kz * zs + col] : T2{0, 0}; };
    auto dst = [&](int kz, int col, T2 v) {
        if (col >= ncol) return;
        const long long gi = base + kz * zs + col;
        if (mode == 0) {
            out[gi] = OT2{(OT)((double)v.x * invN), (OT)((double)v.y * invN)};
        } else {
            T sc;
            if (f == 0) {
                const T kx = kval<T>(g, 0, kx0 + col), kzv = kval<T>(g, 2, kz);
                sc = mN * (kx * kx + kyv * kyv + kzv * kzv);
            } else {
                sc = lN;
            }
            out[gi] = OT2{(OT)(v.x * sc), (OT)(v.y * sc)};
        }
    };
    fft_cols<-1, TX>(g.pz, A, B, src, dst);
}

template <typename T>
void launch_z_fwd(const Geo& g, const Phys& ph, const void* W, void* out, int scale_mode, cudaStream_t s, int nf) {
    using T2 = typename Cx<T>::t;
    const int TX = tuned_cols<T>(g, g.tx_z, g.nz, 2, 128 * 1024);
    const size_t sm = 2 * (size_t)TX * g.nz * sizeof(T2);
    dim3 grid((g.nxh + TX - 1) / TX, g.ny, nf);
    if (scale_mode == 1) {
        PF_TX_SWITCH(TX, set_smem(k_z_fwd<T, T2, TXC>, sm);
                     k_z_fwd<T, T2, TXC><<<grid, kThreads, sm, s>>>(g, ph, reinterpret_cast<const T2*>(W),
                                                                    reinterpret_cast<T2*>(out), 1))
    } else {
        PF_TX_SWITCH(TX, set_smem(k_z_fwd<T, double2, TXC>, sm);
                     k_z_fwd<T, double2, TXC><<<grid, kThreads, sm, s>>>(g, ph, reinterpret_cast<const T2*>(W),
                                                                         reinterpret_cast<double2*>(out),
                                                                         scale_mode))
    }
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

template <typename T, int TX>
__global__ void __launch_bounds__(kThreads) k_z_elastic(Geo g, Phys ph, typename Cx<T>::t* __restrict__ H) {
    PF_SKIP_INACTIVE(g);
    using T2 = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int tile = TX * g.nz;
    T2* slot[3];
    slot[0] = reinterpret_cast<T2*>(smraw);
    slot[1] = slot[0] + tile;
    slot[2] = slot[1] + tile;
    T2* E = slot[2] + tile;
    const int ky = blockIdx.y, kx0 = blockIdx.x * TX;
    const int ncol = min(TX, g.nxh - kx0);
    const long long rowoff = (long long)ky * g.nxh + kx0;
    const long long zs = (long long)g.ny * g.nxh;
    const bool nst_even = (g.pz.nst % 2) == 0;
    // forward transforms: global -> field slot (middle stages ping-pong with E
    // so that the last stage reads E and writes the slot)
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        T2* S = slot[f];
        const long long fb = (long long)f * g.NK + rowoff;
        auto src = [&](int kz, int col) -> T2 { return col < ncol ? H[fb + kz * zs + col] : T2{0, 0}; };
        auto dst = [&](int kz, int col, T2 v) { S[kz * TX + col] = v; };
        if (nst_even)
            fft_cols<-1, TX>(g.pz, E, S, src, dst);
        else
            fft_cols<-1, TX>(g.pz, S, E, src, dst);
        __syncthreads();
    }
    const T invN = (T)(1.0 / (double)g.N);
    const PhysT<T> pt(ph);
    const T kyv = kval<T>(g, 1, ky);
    for (int r = threadIdx.x; r < tile; r += blockDim.x) {
        const int col = r & (TX - 1), kz = r / TX;
        if (col >= ncol) continue;
        T Bm[3][3];
        elastic_kernel<T>(pt, kval<T>(g, 0, kx0 + col), kyv, kval<T>(g, 2, kz), Bm);
        const T2 h0 = slot[0][r], h1 = slot[1][r], h2 = slot[2][r];
        slot[0][r] = T2{(Bm[0][0] * h0.x + Bm[0][1] * h1.x + Bm[0][2] * h2.x) * invN,
                        (Bm[0][0] * h0.y + Bm[0][1] * h1.y + Bm[0][2] * h2.y) * invN};
        slot[1][r] = T2{(Bm[1][0] * h0.x + Bm[1][1] * h1.x + Bm[1][2] * h2.x) * invN,
                        (Bm[1][0] * h0.y + Bm[1][1] * h1.y + Bm[1][2] * h2.y) * invN};
        slot[2][r] = T2{(Bm[2][0] * h0.x + Bm[2][1] * h1.x + Bm[2][2] * h2.x) * invN,
                        (Bm[2][0] * h0.y + Bm[2][1] * h1.y + Bm[2][2] * h2.y) * invN};
    }
    __syncthreads();
    // inverse transforms: field slot -> global (stage 0 reads the slot and
    // writes E)
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        T2* S = slot[f];
        const long long fb = (long long)f * g.NK + rowoff;
        auto src = [&](int kz, int col) -> T2 { return S[kz * TX + col]; };
        auto dst = [&](int kz, int col, T2 v) {
            if (col < ncol) H[fb + kz * zs + col] = v;
        };
        fft_cols<+1, TX>(g.pz, E, S, src, dst);
        __syncthreads();
    }
}

template <typename T>
void launch_z_elastic(const Geo& g, const Phys& ph, void* H, cudaStream_t s) {
    using T2 = typename Cx<T>::t;
    const int TX = tuned_cols<T>(g, g.tx_el, g.nz, 4, 128 * 1024);
    const size_t sm = 4 * (size_t)TX * g.nz * sizeof(T2);
    dim3 grid((g.nxh + TX - 1) / TX, g.ny, 1);
    PF_TX_SWITCH(TX, set_smem(k_z_elastic<T, TXC>, sm);
                 k_z_elastic<T, TXC><<<grid, kThreads, sm, s>>>(g, ph, reinterpret_cast<T2*>(H)))
}

// ---------------------------------------------------------------------------
// z pass: step completion, embedded local error, inverse FFT of the error
//   y_n = y + sum_i (dt b^I_i) lambda z_i + (dt b^E_i) f^E_i
//   LTE = sum_i (dt (b-bt)^I_i) lambda z_i + (dt (b-bt)^E_i) f^E_i
// ---------------------------------------------------------------------------
template <typename T, int TX>
__global__ void __launch_bounds__(kThreads) k_z_final(Geo g, Phys ph, const double2* __restrict__ y, StageTerms bt,
                                                      StageTerms dt, int want_lte, double2* __restrict__ ynew,
                                                      typename Cx<T>::t* __restrict__ W) {
    PF_SKIP_INACTIVE(g);
    using T2 = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smraw[];
    T2* A = reinterpret_cast<T2*>(smraw);
    T2* B = A + TX * g.nz;
    const int f = blockIdx.z, ky = blockIdx.y, kx0 = blockIdx.x * TX;
    const int ncol = min(TX, g.nxh - kx0);
    const long long base = (long long)f * g.NK + (long long)ky * g.nxh + kx0;
    const long long zs = (long long)g.ny * g.nxh;
    const double kyv = g.ky[ky];
    auto combine = [&](int kz, int col) -> T2 {
        if (col >= ncol) return T2{0, 0};
        const long long gi = base + kz * zs + col;
        const double lam = lam_at(g, ph, f, gi, g.kx[kx0 + col], kyv, g.kz[kz]);
        double2 r = y[gi];
        double2 l = make_double2(0.0, 0.0);
        double2 zr = make_double2(0.0, 0.0), zl = make_double2(0.0, 0.0);  // times lambda below
        DS2 rs, ls;
#pragma unroll
        for (int j = 0; j < kMaxStages; ++j) {
            if (j < bt.n) {
                const bool bI = (bt.mI >> j) & 1u, bE = (bt.mE >> j) & 1u;
                const bool lI = want_lte && ((dt.mI >> j) & 1u), lE = want_lte && ((dt.mE >> j) & 1u);
                if (bI || lI) {
                    const double2 zj = bt.z[j][gi];
                    if (bI) axpy(zr, cI_of(bt, j), zj);
                    if (lI) axpy(zl, cI_of(dt, j), zj);
                }
                if (bE || lE) {
                    if (sizeof(T) == 4) {
                        const float2 fj = reinterpret_cast<const float2*>(bt.f[j])[gi];
                        if (bE) rs.add(cEh_of(bt, j), cEl_of(bt, j), fj);
                        if (lE) ls.add(cEh_of(dt, j), cEl_of(dt, j), fj);
                    } else {
                        const double2 fj = load_f<T2>(bt.f[j], gi);
                        if (bE) axpy(r, cE_of(bt, j), fj);
                        if (lE) axpy(l, cE_of(dt, j), fj);
                    }
                }
            }
        }
        axpy(r, lam, zr);
        axpy(l, lam, zl);
        if (sizeof(T) == 4) {
            rs.flush(r);
            ls.flush(l);
        }
        ynew[gi] = r;
        return narrow<T2>(l);
    };
    if (!want_lte) {
        for (int e = threadIdx.x; e < TX * g.nz; e += blockDim.x) combine(e / TX, e & (TX - 1));
        return;
    }
    auto dst = [&](int kz, int col, T2 v) {
        if (col < ncol) W[base + kz * zs + col] = v;
    };
    fft_cols<+1, TX>(g.pz, A, B, combine, dst);
}

template <typename T>
void launch_z_final(const Geo& g, const Phys& ph, const double2* y, const StageTerms& bterm, const StageTerms& dterm,
                    int want_lte, double2* ynew, void* W, cudaStream_t s) {
    using T2 = typename Cx<T>::t;
    const int TX = tuned_cols<T>(g, g.tx_z, g.nz, 2, 128 * 1024);
    const size_t sm = 2 * (size_t)TX * g.nz * sizeof(T2);
    dim3 grid((g.nxh + TX - 1) / TX, g.ny, 4);
    PF_TX_SWITCH(TX, set_smem(k_z_final<T, TXC>, sm);
                 k_z_final<T, TXC><<<grid, kThreads, sm, s>>>(g, ph, y, bterm, dterm, want_lte, ynew,
                                                              reinterpret_cast<T2*>(W)))
}

// ---------------------------------------------------------------------------
// x passes: packed real transforms with the real-space physics fused in.
// Two consecutive rows (y, y+1) of one field share one complex line
// z = a + i b; C2R packs Z_k = A_k + i B_k (Hermitian extension for k > n/2,
// imaginary parts of DC and Nyquist dropped), R2C unpacks
// A_k = (Z_k + conj Z_{n-k})/2, B_k = (Z_k - conj Z_{n-k})/(2i).
// ---------------------------------------------------------------------------
struct Pt {
    // real-space physics at one point (Sec. 4.1); returns q and g_v
    template <typename T>
    __device__ __forceinline__ static void rhs(const PhysT<T>& pt, T X, const T* p, const T* e, T& q, T* gv) {
        T h[3], hp[3];
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            const T f = p[v];
            h[v] = f * f * f * ((T)6 * f * f - (T)15 * f + (T)10);
            hp[v] = (T)30 * f * f * ((T)1 - f) * ((T)1 - f);
        }
        const T H = h[0] + h[1] + h[2];
        const T Bv = pt.Bv, Bm = pt.Bm;
        const T denom = H * pt.inv2Av + ((T)1 - H) * pt.inv2Am;
        const T mu = (X - H * Bv - ((T)1 - H) * Bm) / denom;
        const T Xm = mu * pt.inv2Am + Bm;
        const T Xv = mu * pt.inv2Av + Bv;
        const T fm = pt.A0m + pt.Am * (Xm - Bm) * (Xm - Bm);
        const T fv = pt.A0v + pt.Av * (Xv - Bv) * (Xv - Bv);
        const T drive = fv - fm - mu * (Xv - Xm);
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            const T f = p[v];
            T d = pt.wb2 * f * ((T)1 - f) * ((T)1 - (T)2 * f);
#pragma unroll
            for (int qq = 0; qq < 3; ++qq)
                if (qq != v) {
                    const T sl = fmin((T)1, fmax((T)-1, f * p[qq] * pt.ie));
                    d += pt.w[v][qq] * sl * p[qq];
                }
            gv[v] = d + hp[v] * drive + hp[v] * e[v];
        }
        q = mu - pt.twoAm * X;
    }
};

template <typename T>
__device__ __forceinline__ T hfun(T f) { return f * f * f * ((T)6 * f * f - (T)15 * f + (T)10); }

// load F packed lines (C2R input) of row pairs [rp0, rp0+P) into S
template <typename T2>
__device__ __forceinline__ void c2r_load(const Geo& g, const T2* __restrict__ in, int F, int P, int rp0, int npairs,
                                         T2* S, int ls) {
    const int nx = g.nx, nh = nx / 2;
    const FastDiv dnx((unsigned)nx, g.mul_nx);
    for (int e = threadIdx.x; e < P * F * nx; e += blockDim.x) {
        const int line = (int)dnx.div((unsigned)e), x = e - line * nx, rp = line / F, f = line - rp * F;
        T2 Z = T2{0, 0};
        if (rp0 + rp < npairs) {
            const long long row = 2LL * (rp0 + rp);
            const int k = x <= nh ? x : nx - x;
            const T2* base = in + (long long)f * g.NK + row * g.nxh + k;
            T2 a = base[0], b = base[g.nxh];
            if (k == 0 || k == nh) {
                a.y = 0;
                b.y = 0;
            }
            if (x <= nh)
                Z = T2{a.x - b.y, a.y + b.x};
            else
                Z = T2{a.x + b.y, b.x - a.y};
        }
        S[line * ls + x] = Z;
    }
}

template <typename T2>
__device__ __forceinline__ void r2c_store(const Geo& g, const T2* S, int ls, int F, int P, int rp0, int npairs,
                                          T2* __restrict__ out) {
    using T = decltype(T2{}.x);
    const int nx = g.nx, nxh = g.nxh;
    const FastDiv dnh((unsigned)nxh, g.mul_nxh);
    for (int e = threadIdx.x; e < P * F * nxh; e += blockDim.x) {
        const int line = (int)dnh.div((unsigned)e), k = e - line * nxh, rp = line / F, f = line - rp * F;
        if (rp0 + rp >= npairs) continue;
        const T2 Zk = S[line * ls + k];
        const T2 Zm = S[line * ls + (k == 0 ? 0 : nx - k)];
        const T half = (T)0.5;
        const T2 A = T2{(Zk.x + Zm.x) * half, (Zk.y - Zm.y) * half};
        const T2 B = T2{(Zk.y + Zm.y) * half, (Zm.x - Zk.x) * half};
        const long long row = 2LL * (rp0 + rp);
        T2* base = out + (long long)f * g.NK + row * nxh + k;
        base[0] = A;
        base[nxh] = B;
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_x_pass(Geo g, Phys ph, int mode, const typename Cx<T>::t* __restrict__ in,
                                                     typename Cx<T>::t* __restrict__ out, T* __restrict__ R,
                                                     const T* __restrict__ Rin, double* __restrict__ partials,
                                                     double rtol, double atol, const double* __restrict__ real_in,
                                                     double* __restrict__ real_out, int P) {
    PF_SKIP_INACTIVE(g);
    using T2 = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nx = g.nx;
    const int ls = nx;
    const FastDiv dnx((unsigned)nx, g.mul_nx);
    const PhysT<T> pt(ph);
    const int npairs = g.nz * g.ny / 2;
    const int rp0 = blockIdx.x * P;
    T2* S0 = reinterpret_cast<T2*>(smraw);
    T2* S1 = S0 + 4 * P * nx;
    __shared__ double red[kThreads / 32];

    // ---- input: C2R of the incoming half-spectrum lines, or packed real rows
    int Fin = 0;
    if (mode == XM_PHYS1 || mode == XM_WRMS || mode == XM_C2R_REAL || mode == XM_ENERGY) Fin = 4;
    if (mode == XM_PHYS2) Fin = ph.elastic ? 3 : 0;
    T2* RS = S0;  // real-space lines (a + i b)
    if (mode == XM_R2C_REAL) {
        for (int e = threadIdx.x; e < P * 4 * nx; e += blockDim.x) {
            const int line = (int)dnx.div((unsigned)e), x = e - line * nx, rp = line >> 2, f = line & 3;
            T2 Z = T2{0, 0};
            if (rp0 + rp < npairs) {
                const long long row = 2LL * (rp0 + rp);
                const double* b = real_in + (long long)f * g.N + row * nx + x;
                Z = T2{(T)b[0], (T)b[nx]};
            }
            S0[line * ls + x] = Z;
        }
        __syncthreads();
        T2* res = fft_lines<-1, false>(S0, S1, g.px, 4 * P, 1, ls);
        r2c_store(g, res, ls, 4, P, rp0, npairs, out);
        return;
    }
    if (Fin > 0) {
        c2r_load(g, in, Fin, P, rp0, npairs, S0, ls);
        __syncthreads();
        RS = fft_lines<+1, false>(S0, S1, g.px, Fin * P, 1, ls);
    }
    T2* OS = (RS == S0) ? S1 : S0;  // output lines

    if (mode == XM_C2R_REAL) {
        for (int e = threadIdx.x; e < P * 4 * nx; e += blockDim.x) {
            const int line = (int)dnx.div((unsigned)e), x = e - line * nx, rp = line >> 2, f = line & 3;
            if (rp0 + rp >= npairs) continue;
            const long long row = 2LL * (rp0 + rp);
            const T2 z = RS[line * ls + x];
            double* b = real_out + (long long)f * g.N + row * nx + x;
            b[0] = (double)z.x;
            b[nx] = (double)z.y;
        }
        return;
    }

    if (mode == XM_WRMS) {
        double acc = 0.0;
        for (int e = threadIdx.x; e < P * 4 * nx; e += blockDim.x) {
            const int line = (int)dnx.div((unsigned)e), x = e - line * nx, rp = line >> 2, f = line & 3;
            if (rp0 + rp >= npairs) continue;
            const long long row = 2LL * (rp0 + rp);
            const T2 z = RS[line * ls + x];
            const T* yr = Rin + (long long)f * g.N + row * nx + x;
            // weighted error w_i * LTE_i formed in the compute type (the
            // error and y_{n-1} are already compute-type fields); squares
            // accumulated in FP64
            const T rt = (T)rtol, at = (T)atol;
            const T a = z.x / (rt * fabs(yr[0]) + at), b = z.y / (rt * fabs(yr[nx]) + at);
            if (sizeof(T) == 4) {
                const double da = f2d_bits((float)a), db = f2d_bits((float)b);
                acc = fma(da, da, acc);
                acc = fma(db, db, acc);
            } else {
                acc += (double)a * (double)a + (double)b * (double)b;
            }
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
            partials[blockIdx.x] = s;
        }
        return;
    }

    // ---- pointwise physics: 2 rows per line, all fields of a point together
    int Fout = 0;
    double eacc = 0.0;
    const bool full_rhs = (mode == XM_PHYS2) || (mode == XM_PHYS1 && !ph.elastic);
    for (int e = threadIdx.x; e < P * nx; e += blockDim.x) {
        const int rp = (int)dnx.div((unsigned)e), x = e - rp * nx;
        if (rp0 + rp >= npairs) continue;
        const long long row = 2LL * (rp0 + rp);
        T Xr[2], pr[2][3], er[2][3];
        if (mode == XM_PHYS2) {
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                const T* b = Rin + (long long)f * g.N + row * nx + x;
                if (f == 0) {
                    Xr[0] = b[0];
                    Xr[1] = b[nx];
                } else {
                    pr[0][f - 1] = b[0];
                    pr[1][f - 1] = b[nx];
                }
            }
#pragma unroll
            for (int v = 0; v < 3; ++v) {
                if (ph.elastic) {
                    const T2 z = RS[(rp * 3 + v) * ls + x];
                    er[0][v] = z.x;
                    er[1][v] = z.y;
                } else {
                    er[0][v] = 0;
                    er[1][v] = 0;
                }
            }
        } else {
            const T2 zX = RS[(rp * 4 + 0) * ls + x];
            Xr[0] = zX.x;
            Xr[1] = zX.y;
#pragma unroll
            for (int v = 0; v < 3; ++v) {
                const T2 z = RS[(rp * 4 + 1 + v) * ls + x];
                pr[0][v] = z.x;
                pr[1][v] = z.y;
                er[0][v] = 0;
                er[1][v] = 0;
            }
            if (mode == XM_PHYS1 && R) {
#pragma unroll
                for (int f = 0; f < 4; ++f) {
                    T* b = R + (long long)f * g.N + row * nx + x;
                    b[0] = f == 0 ? Xr[0] : pr[0][f - 1];
                    b[nx] = f == 0 ? Xr[1] : pr[1][f - 1];
                }
            }
        }
        if (full_rhs) {
            T q[2], gv[2][3];
#pragma unroll
            for (int r = 0; r < 2; ++r) Pt::rhs<T>(pt, Xr[r], pr[r], er[r], q[r], gv[r]);
            OS[(rp * 4 + 0) * ls + x] = T2{q[0], q[1]};
#pragma unroll
            for (int v = 0; v < 3; ++v) OS[(rp * 4 + 1 + v) * ls + x] = T2{gv[0][v], gv[1][v]};
        } else {
            // h(phi_v) lines for the elastic contraction (and the local energy)
#pragma unroll
            for (int v = 0; v < 3; ++v) OS[(rp * 3 + v) * ls + x] = T2{hfun(pr[0][v]), hfun(pr[1][v])};
            if (mode == XM_ENERGY) {
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const double X = (double)Xr[r];
                    double p[3], h[3];
                    for (int v = 0; v < 3; ++v) {
                        p[v] = (double)pr[r][v];
                        h[v] = p[v] * p[v] * p[v] * (6.0 * p[v] * p[v] - 15.0 * p[v] + 10.0);
                    }
                    const double H = h[0] + h[1] + h[2];
                    const double denom = H * ph.inv2Av + (1.0 - H) * ph.inv2Am;
                    const double mu = (X - H * ph.Bv - (1.0 - H) * ph.Bm) / denom;
                    const double Xm = mu * ph.inv2Am + ph.Bm, Xv = mu * ph.inv2Av + ph.Bv;
                    const double fm = ph.A0m + ph.Am * (Xm - ph.Bm) * (Xm - ph.Bm);
                    const double fv = ph.A0v + ph.Av * (Xv - ph.Bv) * (Xv - ph.Bv);
                    double loc = 0.0;
                    for (int v = 0; v < 3; ++v) loc += ph.wbar * p[v] * p[v] * (1.0 - p[v]) * (1.0 - p[v]);
                    const double e = ph.pair_eps;
                    const double pr[3] = {p[0] * p[1], p[0] * p[2], p[1] * p[2]};
                    const double wv[3] = {ph.w[0][1], ph.w[0][2], ph.w[1][2]};
                    for (int k = 0; k < 3; ++k) {
                        const double ax = fabs(pr[k]);
                        loc += wv[k] * (ax < e ? pr[k] * pr[k] / (2.0 * e) : ax - 0.5 * e);
                    }
                    loc += H * fv + (1.0 - H) * fm;
                    eacc += loc;
                }
            }
        }
    }
    Fout = full_rhs ? 4 : 3;
    if (mode == XM_ENERGY) {
        for (int o = 16; o > 0; o >>= 1) eacc += __shfl_xor_sync(0xffffffffu, eacc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = eacc;
    }
    __syncthreads();
    if (mode == XM_ENERGY && threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
        partials[blockIdx.x] = s;
    }
    T2* res = fft_lines<-1, false>(OS, RS, g.px, Fout * P, 1, ls);
    r2c_store(g, res, ls, Fout, P, rp0, npairs, out);
}

template <typename T>
static int x_rows(const Geo& g) {
    using T2 = typename Cx<T>::t;
    int Pmax = (int)(64 * 1024 / (8 * (size_t)g.nx * sizeof(T2)));
    if (Pmax < 1) Pmax = 1;
    if (Pmax > 16) Pmax = 16;
    if (g.rp > 0) {
        int P = 1;
        while (P * 2 <= g.rp && P * 2 <= Pmax) P *= 2;
        return P;
    }
    int P = Pmax;
    const int npairs = g.nz * g.ny / 2;
    // keep at least ~2 waves of CTAs on 152 SMs
    while (P > 1 && (npairs + P - 1) / P < 304) P >>= 1;
    return P;
}

// plan from an explicit radix order (each radix in {2,3,4,5,8}, product n)
bool make_axis_plan_radices(int n, const int* rad, int nr, AxisPlan& p) {
    if (nr < 1 || nr > kMaxRadices) return false;
    long long prod = 1;
    for (int s = 0; s < nr; ++s) {
        if (rad[s] != 2 && rad[s] != 3 && rad[s] != 4 && rad[s] != 5 && rad[s] != 8) return false;
        prod *= rad[s];
    }
    if (prod != n) return false;
    p.n = n;
    p.nst = nr;
    unsigned Ns = 1;
    for (int s = 0; s < nr; ++s) {
        p.rad[s] = rad[s];
        p.mulm[s] = magic_u32((unsigned)(n / rad[s]));
        p.mulN[s] = magic_u32(Ns);
        Ns *= (unsigned)rad[s];
    }
    return true;
}

// default schedule: radix-8 stages first, then a 4 (or 4*4 instead of 8*2)
// or 2, then the 3s and 5s
bool make_axis_plan(int n, AxisPlan& p) {
    int m = n, a = 0, b = 0, c = 0;
    while (m % 2 == 0) { m /= 2; ++a; }
    while (m % 3 == 0) { m /= 3; ++b; }
    while (m % 5 == 0) { m /= 5; ++c; }
    if (m != 1) return false;
    int r[kMaxRadices + 8];
    int nr = 0;
    int n8 = a / 3;
    const int rem = a % 3;
    bool two4 = false;
    if (rem == 1 && n8 > 0) {
        --n8;
        two4 = true;
    }
    for (int i = 0; i < n8; ++i) r[nr++] = 8;
    if (two4) {
        r[nr++] = 4;
        r[nr++] = 4;
    } else if (rem == 2) {
        r[nr++] = 4;
    } else if (rem == 1) {
        r[nr++] = 2;
    }
    for (int i = 0; i < b; ++i) r[nr++] = 3;
    for (int i = 0; i < c; ++i) r[nr++] = 5;
    return make_axis_plan_radices(n, r, nr, p);
}

int x_pass_blocks(const Geo& g, int f64) {
    const int P = f64 ? x_rows<double>(g) : x_rows<float>(g);
    const int npairs = g.nz * g.ny / 2;
    return (npairs + P - 1) / P;
}

template <typename T>
void launch_x_pass(const Geo& g, const Phys& ph, int mode, const void* in, void* out, void* R, const void* Rin,
                   double* partials, double rtol, double atol, const double* real_in, double* real_out,
                   cudaStream_t s) {
    using T2 = typename Cx<T>::t;
    const int P = x_rows<T>(g);
    const size_t sm = 2 * 4 * (size_t)P * g.nx * sizeof(T2);
    set_smem(k_x_pass<T>, sm);
    const int npairs = g.nz * g.ny / 2;
    const int nb = (npairs + P - 1) / P;
    k_x_pass<T><<<nb, kThreads, sm, s>>>(g, ph, mode, reinterpret_cast<const T2*>(in), reinterpret_cast<T2*>(out),
                                         reinterpret_cast<T*>(R), reinterpret_cast<const T*>(Rin), partials, rtol,
                                         atol, real_in, real_out, P);
}

// ---------------------------------------------------------------------------
// pointwise kernels (FP64)
// ---------------------------------------------------------------------------
__global__ void k_stage_pointwise(Geo g, Phys ph, const double2* __restrict__ y, StageTerms st, int fe32,
                                  double2* __restrict__ zout) {
    PF_SKIP_INACTIVE(g);
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

void launch_stage_pointwise(const Geo& g, const Phys& ph, const double2* y, const StageTerms& st, int fe_is_f32,
                            double2* zout, cudaStream_t s) {
    k_stage_pointwise<<<152 * 8, 256, 0, s>>>(g, ph, y, st, fe_is_f32, zout);
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

__global__ void k_lambda_table(Geo g, Phys ph, double* __restrict__ lam) {
    const long long total = 4LL * g.NK;
    for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < total;
         gi += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(gi / g.NK);
        const long long q = gi % g.NK;
        const int kx = (int)(q % g.nxh);
        const int ky = (int)((q / g.nxh) % g.ny);
        const int kz = (int)(q / ((long long)g.nxh * g.ny));
        lam[gi] = lambda_k(ph, f, g.kx[kx], g.ky[ky], g.kz[kz]);
    }
}

void launch_lambda_table(const Geo& g, const Phys& ph, double* lam, cudaStream_t s) {
    k_lambda_table<<<152 * 8, 256, 0, s>>>(g, ph, lam);
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
    }
    c.gamma = gam;
    c.qgamma = qgam;
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

// y <- y_new for an accepted attempt
__global__ void k_batch_accept(Geo g, const MemberCtl* __restrict__ ctl, const double2* __restrict__ ynew,
                               double2* __restrict__ y) {
    if (!ctl->accepted_now) return;
    const long long total = 4LL * g.NK;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x)
        y[i] = ynew[i];
}

void launch_batch_prep(const BatchConst& bc, MemberCtl* ctl, StageCoefDev* coef, cudaStream_t s) {
    k_batch_prep<<<1, 32, 0, s>>>(bc, ctl, coef);
}
void launch_batch_ctl(const BatchConst& bc, MemberCtl* ctl, const double* wrms_sum, double scale, cudaStream_t s) {
    k_batch_ctl<<<1, 32, 0, s>>>(bc, ctl, wrms_sum, scale);
}
void launch_batch_accept(const Geo& g, const MemberCtl* ctl, const double2* ynew, double2* y, cudaStream_t s) {
    k_batch_accept<<<152 * 4, 256, 0, s>>>(g, ctl, ynew, y);
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
            const PhysT<double> pt(ph);
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

// explicit instantiations
#define PF_INST(T)                                                                                                 \
    template void launch_z_stage<T>(const Geo&, const Phys&, const double2*, const StageTerms&, double2*, void*,   \
                                    cudaStream_t);                                                                 \
    template void launch_y_pass<T>(const Geo&, void*, int, int, cudaStream_t);                                    \
    template void launch_x_pass<T>(const Geo&, const Phys&, int, const void*, void*, void*, const void*, double*,  \
                                   double, double, const double*, double*, cudaStream_t);                          \
    template void launch_z_elastic<T>(const Geo&, const Phys&, void*, cudaStream_t);                               \
    template void launch_z_fwd<T>(const Geo&, const Phys&, const void*, void*, int, cudaStream_t, int);                 \
    template void launch_z_final<T>(const Geo&, const Phys&, const double2*, const StageTerms&, const StageTerms&, \
                                    int, double2*, void*, cudaStream_t);
PF_INST(double)
PF_INST(float)

}  // namespace pf
