// Fourier neural operator surrogate: forward, backward and Adam, all on the
// GPU (FP32 activations and accumulation; the spectral weights are read in
// BF16 unless the FP32 checking mode is selected).
//
//   a_0 = P x + p
//   for each layer l: A = F_K(a_l) (truncated DFT, kx < m, |ky|,|kz| < m),
//                     O = W_l A per mode (complex C x C),
//                     s = (1/N) Re sum_K w_kx O e^{ik.r},
//                     z = V_l a_l + v_l + s,  a_{l+1} = GELU(z) (not after the last layer)
//   h = GELU(Q1 a_L + q1), out = Q2 h + q2
//
// Truncated transforms and their adjoints are small dense contractions along
// one axis (kernel k_axis with precomputed complex matrices).  The per-mode
// channel mix is a batch-1 32x32 complex matvec per retained mode: it streams
// the weights once per pass (weight-bandwidth bound), so it runs on CUDA cores
// from BF16 storage rather than through the tensor cores.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "pf.h"
#include "pf_internal.h"

using namespace pf;

int pf_ctx_grid(pf_ctx* c, pf_grid* g);

namespace {

constexpr int kT = 256;

struct FnoDims {
    int nx, ny, nz, C, m, H, L, cin;
    long long N;
    int K;  // (2m)(2m)m retained modes
};

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_g(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// out[o][k][i] (=|+=) sum_j M[k][j] in[o][j][i]; complex M [nk][nj]
template <bool IN_REAL, bool OUT_REAL, bool ACCUM>
__global__ void k_axis(const void* __restrict__ inp, void* __restrict__ outp, const float2* __restrict__ M, int nk,
                       int nj, long long n_outer, int n_inner) {
    extern __shared__ float2 Ms[];
    for (int e = threadIdx.x; e < nk * nj; e += blockDim.x) Ms[e] = M[e];
    __syncthreads();
    const long long total = n_outer * nk * n_inner;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx % n_inner);
        const long long ok = idx / n_inner;
        const int k = (int)(ok % nk);
        const long long o = ok / nk;
        float ar = 0.f, ai = 0.f;
        const long long ib = o * nj * (long long)n_inner + i;
        for (int j = 0; j < nj; ++j) {
            const float2 m = Ms[k * nj + j];
            if (IN_REAL) {
                const float v = reinterpret_cast<const float*>(inp)[ib + (long long)j * n_inner];
                ar += m.x * v;
                ai += m.y * v;
            } else {
                const float2 v = reinterpret_cast<const float2*>(inp)[ib + (long long)j * n_inner];
                ar += m.x * v.x - m.y * v.y;
                ai += m.x * v.y + m.y * v.x;
            }
        }
        const long long ob = (o * nk + k) * (long long)n_inner + i;
        if (OUT_REAL) {
            float* out = reinterpret_cast<float*>(outp);
            out[ob] = ACCUM ? out[ob] + ar : ar;
        } else {
            float2* out = reinterpret_cast<float2*>(outp);
            out[ob] = ACCUM ? make_float2(out[ob].x + ar, out[ob].y + ai) : make_float2(ar, ai);
        }
    }
}

// spectral weight (re, im) of mode k, row c, column d
__device__ __forceinline__ float2 wget(const float2* w32, const __nv_bfloat162* w16, long long e) {
    if (w16) {
        const __nv_bfloat162 b = w16[e];
        return make_float2(__bfloat162float(b.x), __bfloat162float(b.y));
    }
    return w32[e];
}

// O[c][k] = sum_d W[k][c][d] A[d][k]
__global__ void k_mix(const float2* __restrict__ A, float2* __restrict__ O, const float2* __restrict__ w32,
                      const __nv_bfloat162* __restrict__ w16, int C, int K) {
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < (long long)C * K;
         idx += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(idx % K), c = (int)(idx / K);
        float ar = 0.f, ai = 0.f;
        const long long wb = ((long long)k * C + c) * C;
        for (int d = 0; d < C; ++d) {
            const float2 w = wget(w32, w16, wb + d);
            const float2 a = A[(long long)d * K + k];
            ar += w.x * a.x - w.y * a.y;
            ai += w.x * a.y + w.y * a.x;
        }
        O[idx] = make_float2(ar, ai);
    }
}

// backward of the mix: GA[d][k] = sum_c conj(W[k][c][d]) GO[c][k];
// GW[k][c][d] = GO[c][k] conj(A[d][k])
__global__ void k_mix_bwd(const float2* __restrict__ GO, const float2* __restrict__ A, float2* __restrict__ GA,
                          float2* __restrict__ GW, const float2* __restrict__ w32,
                          const __nv_bfloat162* __restrict__ w16, int C, int K) {
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < (long long)C * K;
         idx += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(idx % K), d = (int)(idx / K);
        float ar = 0.f, ai = 0.f;
        const float2 a = A[(long long)d * K + k];
        for (int c = 0; c < C; ++c) {
            const long long e = ((long long)k * C + c) * C + d;
            const float2 w = wget(w32, w16, e);
            const float2 g = GO[(long long)c * K + k];
            ar += w.x * g.x + w.y * g.y;  // conj(w) g
            ai += w.x * g.y - w.y * g.x;
            GW[e] = make_float2(g.x * a.x + g.y * a.y, g.y * a.x - g.x * a.y);  // g conj(a)
        }
        GA[idx] = make_float2(ar, ai);
    }
}

// y[a][p] = sum_b Mw[a][b] x[b][p] + bias[a] (+ add[a][p]); optional GELU
// output, pre-activation kept in zout
__global__ void k_dense(const float* __restrict__ x, float* __restrict__ y, float* __restrict__ zout,
                        const float* __restrict__ Mw, const float* __restrict__ bias, const float* __restrict__ add,
                        int A, int B, long long N, int act) {
    extern __shared__ float sm[];
    for (int e = threadIdx.x; e < A * B + A; e += blockDim.x) sm[e] = e < A * B ? Mw[e] : bias[e - A * B];
    __syncthreads();
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
        for (int a = 0; a < A; ++a) {
            float acc = sm[A * B + a];
            for (int b = 0; b < B; ++b) acc += sm[a * B + b] * x[(long long)b * N + p];
            if (add) acc += add[(long long)a * N + p];
            if (zout) zout[(long long)a * N + p] = acc;
            y[(long long)a * N + p] = act ? gelu_f(acc) : acc;
        }
    }
}

// dx[b][p] (=|+=) sum_a Mw[a][b] dy[a][p]
__global__ void k_dense_t(const float* __restrict__ dy, float* __restrict__ dx, const float* __restrict__ Mw, int A,
                          int B, long long N, int accum) {
    extern __shared__ float sm[];
    for (int e = threadIdx.x; e < A * B; e += blockDim.x) sm[e] = Mw[e];
    __syncthreads();
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
        for (int b = 0; b < B; ++b) {
            float acc = 0.f;
            for (int a = 0; a < A; ++a) acc += sm[a * B + b] * dy[(long long)a * N + p];
            const long long i = (long long)b * N + p;
            dx[i] = accum ? dx[i] + acc : acc;
        }
    }
}

// g[i] *= GELU'(z[i])
__global__ void k_gelu_bwd(float* __restrict__ g, const float* __restrict__ z, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        g[i] *= gelu_g(z[i]);
}

// per-block partial sums of G[a][b] = sum_p U[a][p] V[b][p] (V = ones when
// null: column sums of U), written to part[block][a][b]
constexpr int kCh = 32;
__global__ void k_outer_partial(const float* __restrict__ U, const float* __restrict__ V, int A, int B, long long N,
                                float* __restrict__ part) {
    extern __shared__ float sm[];
    float* su = sm;
    float* sv = sm + A * kCh;
    const int E = A * B;
    float acc[16];
    for (int q = 0; q < 16; ++q) acc[q] = 0.f;
    const long long per = (N + gridDim.x - 1) / gridDim.x;
    const long long p0 = blockIdx.x * per, p1 = min(N, p0 + per);
    for (long long pc = p0; pc < p1; pc += kCh) {
        const int np = (int)min((long long)kCh, p1 - pc);
        __syncthreads();
        for (int e = threadIdx.x; e < A * kCh; e += blockDim.x) {
            const int a = e / kCh, q = e % kCh;
            su[e] = q < np ? U[(long long)a * N + pc + q] : 0.f;
        }
        for (int e = threadIdx.x; e < B * kCh; e += blockDim.x) {
            const int b = e / kCh, q = e % kCh;
            sv[e] = q < np ? (V ? V[(long long)b * N + pc + q] : 1.f) : 0.f;
        }
        __syncthreads();
        for (int q = 0; q < 16; ++q) {
            const int e = threadIdx.x + q * blockDim.x;
            if (e >= E) break;
            const int a = e / B, b = e % B;
            float s = 0.f;
            for (int t = 0; t < kCh; ++t) s += su[a * kCh + t] * sv[b * kCh + t];
            acc[q] += s;
        }
    }
    for (int q = 0; q < 16; ++q) {
        const int e = threadIdx.x + q * blockDim.x;
        if (e < E) part[(long long)blockIdx.x * E + e] = acc[q];
    }
}

// G[e] = sum_blocks part[blk][e] (fixed order)
__global__ void k_sum_partials(const float* __restrict__ part, int nblk, int E, float* __restrict__ G) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int b = 0; b < nblk; ++b) s += part[(long long)b * E + e];
        G[e] = s;
    }
}

// dout = 2 (out - tgt) / n_el and per-block sums of (out - tgt)^2
__global__ void k_mse(const float* __restrict__ out, const float* __restrict__ tgt, float* __restrict__ dout,
                      long long n, double* __restrict__ part) {
    __shared__ double red[kT / 32];
    double acc = 0.0;
    const float sc = 2.0f / (float)n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float d = out[i] - tgt[i];
        dout[i] = sc * d;
        acc += (double)d * d;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        part[blockIdx.x] = s;
    }
}

__global__ void k_adam(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

__global__ void k_to_bf16(const float2* __restrict__ w, __nv_bfloat162* __restrict__ o, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        o[i] = __floats2bfloat162_rn(w[i].x, w[i].y);
}

// real-space state (FP64, [4][N]) -> normalised FP32 network input
__global__ void k_norm_in(const double* __restrict__ y, float* __restrict__ x, long long N, float4 mean, float4 istd) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 4 * N; i += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(i / N);
        const float mu = f == 0 ? mean.x : f == 1 ? mean.y : f == 2 ? mean.z : mean.w;
        const float is = f == 0 ? istd.x : f == 1 ? istd.y : f == 2 ? istd.z : istd.w;
        x[i] = ((float)y[i] - mu) * is;
    }
}

// proposal: y_real += out * out_std (per channel), in FP64
__global__ void k_apply_delta(double* __restrict__ y, const float* __restrict__ out, long long N, float4 ostd) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 4 * N; i += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(i / N);
        const float s = f == 0 ? ostd.x : f == 1 ? ostd.y : f == 2 ? ostd.z : ostd.w;
        y[i] += (double)(out[i] * s);
    }
}

// per-channel sums over the snapshot pairs (s_t, s_{t+1}) of n_traj
// trajectories of n_snap snapshots [traj][snap][4][N]: sums of x, x^2 of the
// inputs s_t and of d, d^2 of the increments d = s_{t+1} - s_t, in FP64,
// per block (part[block][16])
__global__ void k_pair_stats(const float* __restrict__ snaps, int n_traj, int n_snap, long long N,
                             double* __restrict__ part) {
    __shared__ double red[16][kT / 32];
    double acc[16];
    for (int q = 0; q < 16; ++q) acc[q] = 0.0;
    const long long per_pair = 4 * N;
    const long long total = (long long)n_traj * (n_snap - 1) * per_pair;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long pr = i / per_pair, r = i - pr * per_pair;
        const long long tr = pr / (n_snap - 1), t = pr - tr * (n_snap - 1);
        const int f = (int)(r / N);
        const float* a = snaps + (tr * n_snap + t) * per_pair;
        const double x = a[r], d = (double)(a[r + per_pair] - a[r]);
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (c == f) {
                acc[4 * c + 0] += x;
                acc[4 * c + 1] += x * x;
                acc[4 * c + 2] += d;
                acc[4 * c + 3] += d * d;
            }
    }
    for (int q = 0; q < 16; ++q) {
        double v = acc[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < 16) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[threadIdx.x][w];
        part[(long long)blockIdx.x * 16 + threadIdx.x] = v;
    }
}

// network input x = (s_t - mean) / std and target (s_{t+tau} - s_t) / out_std
__global__ void k_pair_prep(const float* __restrict__ s0, const float* __restrict__ s1, float* __restrict__ x,
                            float* __restrict__ tgt, long long N, float4 mean, float4 istd, float4 iostd) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 4 * N;
         i += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(i / N);
        const float mu = f == 0 ? mean.x : f == 1 ? mean.y : f == 2 ? mean.z : mean.w;
        const float is = f == 0 ? istd.x : f == 1 ? istd.y : f == 2 ? istd.z : istd.w;
        const float io = f == 0 ? iostd.x : f == 1 ? iostd.y : f == 2 ? iostd.z : iostd.w;
        const float a = s0[i];
        x[i] = (a - mu) * is;
        tgt[i] = (s1[i] - a) * io;
    }
}

// per-block sums of ((a - b) w)^2 with w = 1/(rtol |b| + atol) (FP64)
__global__ void k_wrms_dist(const double* __restrict__ a, const double* __restrict__ b, long long n, double rtol,
                            double atol, double* __restrict__ part) {
    __shared__ double red[kT / 32];
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double d = (a[i] - b[i]) / (rtol * fabs(b[i]) + atol);
        acc += d * d;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        part[blockIdx.x] = s;
    }
}

// ---------------------------------------------------------------------------
// Tensor-core forms of the pointwise channel contractions (BF16 mode): the
// dense layers y = W x (+ bias, + add, GELU), their transposes dx = W^T dy,
// and the weight gradients G = U V^T summed over the grid points, as BF16
// mma.sync m16n8k16 with FP32 accumulation.  Each FP32 operand v is split
// into v_hi = bf16(v) and v_lo = bf16(v - v_hi), and the product is formed
// as hi*hi + hi*lo + lo*hi, which keeps about 16 significant bits of both
// operands (the dropped lo*lo term is ~2^-16 relative), so the contractions
// cost the weights' and activations' FP32 copies no accuracy beyond the BF16
// spectral weights of this mode.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
// two FP32 values -> their BF16 leading parts packed (first value in the low
// half) and the BF16 roundings of their remainders
__device__ __forceinline__ void split2(float x0, float x1, unsigned& hi, unsigned& lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
    const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - __bfloat162float(h.x), x1 - __bfloat162float(h.y));
    hi = *reinterpret_cast<const unsigned*>(&h);
    lo = *reinterpret_cast<const unsigned*>(&l);
}
__device__ __forceinline__ void mma3(float (&d)[4], const unsigned (&ah)[4], const unsigned (&al)[4], unsigned bh0,
                                     unsigned bh1, unsigned bl0, unsigned bl1) {
    mma_bf16_16816(d, ah, bh0, bh1);
    mma_bf16_16816(d, ah, bl0, bl1);
    mma_bf16_16816(d, al, bh0, bh1);
}

constexpr int kMmaWarps = 4;

// y[m][p] = act(sum_k W'[m][k] x[k][p] + bias[m] (+ add[m][p])), W' = W (M x K
// = A x B) or, with TRANS, W^T (M x K = B x A; out = accum ? out + . : .).
// MT m-tiles of 16 rows; one warp per 8 consecutive points at a time.
template <int MT, bool TRANS>
__global__ void __launch_bounds__(32 * kMmaWarps) k_dense_mma(const float* __restrict__ x, float* __restrict__ y,
                                                              float* __restrict__ zout, const float* __restrict__ W,
                                                              const float* __restrict__ bias,
                                                              const float* __restrict__ add, int A, int B, long long N,
                                                              int act, int accum) {
    const int M = TRANS ? B : A, K = TRANS ? A : B;
    const int KT = (K + 15) / 16;  // k-tiles of 16 (zero padded)
    extern __shared__ unsigned wsm[];  // per (m-tile, k-tile): 32 lanes x 4 regs, hi then lo
    for (int e = threadIdx.x; e < MT * KT * 32; e += blockDim.x) {
        const int lane = e & 31, tile = e >> 5, mt = tile / KT, kt = tile - mt * KT;
        const int g = lane >> 2, t = lane & 3;
        unsigned* dh = wsm + (size_t)tile * 256 + lane * 4;
        unsigned* dl = dh + 128;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int m = mt * 16 + g + ((r & 1) ? 8 : 0), k = kt * 16 + 2 * t + ((r & 2) ? 8 : 0);
            auto wv = [&](int mm, int kk) -> float {
                if (mm >= M || kk >= K) return 0.f;
                return TRANS ? W[(long long)kk * B + mm] : W[(long long)mm * B + kk];
            };
            split2(wv(m, k), wv(m, k + 1), dh[r], dl[r]);
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
    const long long ntiles = (N + 7) / 8;
    for (long long nt = blockIdx.x * (long long)kMmaWarps + warp; nt < ntiles; nt += (long long)gridDim.x * kMmaWarps) {
        const long long p = nt * 8 + g;  // this lane's point in the B fragment
        float acc[MT][4];
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) acc[mt][0] = acc[mt][1] = acc[mt][2] = acc[mt][3] = 0.f;
        for (int kt = 0; kt < KT; ++kt) {
            float xv[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int k = kt * 16 + 2 * t + (r & 1) + ((r & 2) ? 8 : 0);
                xv[r] = (k < K && p < N) ? x[(long long)k * N + p] : 0.f;
            }
            unsigned bh0, bl0, bh1, bl1;
            split2(xv[0], xv[1], bh0, bl0);
            split2(xv[2], xv[3], bh1, bl1);
#pragma unroll
            for (int mt = 0; mt < MT; ++mt) {
                const unsigned* sh = wsm + (size_t)(mt * KT + kt) * 256 + lane * 4;
                const unsigned ah[4] = {sh[0], sh[1], sh[2], sh[3]};
                const unsigned al[4] = {sh[128], sh[129], sh[130], sh[131]};
                mma3(acc[mt], ah, al, bh0, bh1, bl0, bl1);
            }
        }
        // epilogue: acc[mt][0..1] -> rows mt*16 + g, points nt*8 + 2t + {0,1};
        // acc[mt][2..3] -> rows + 8
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int m = mt * 16 + g + ((r & 2) ? 8 : 0);
                const long long q = nt * 8 + 2 * t + (r & 1);
                if (m >= M || q >= N) continue;
                const long long i = (long long)m * N + q;
                float v = acc[mt][r];
                if (TRANS) {
                    y[i] = accum ? y[i] + v : v;
                } else {
                    v += bias[m];
                    if (add) v += add[i];
                    if (zout) zout[i] = v;
                    y[i] = act ? gelu_f(v) : v;
                }
            }
    }
}

// per-block partial sums of G[a][b] = sum_p U[a][p] V[b][p] (U: A x N, V: B x
// N), K = the grid points; warps split the m-tiles, each holding all NT
// n-tiles of its rows; CTAs split the points.
template <int MTW, int NT>
__global__ void __launch_bounds__(32 * kMmaWarps) k_outer_mma(const float* __restrict__ U, const float* __restrict__ V,
                                                              int A, int B, long long N, float* __restrict__ part) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
    const int MT = (A + 15) / 16;
    float acc[MTW][NT][4];
#pragma unroll
    for (int i = 0; i < MTW; ++i)
#pragma unroll
        for (int j = 0; j < NT; ++j) acc[i][j][0] = acc[i][j][1] = acc[i][j][2] = acc[i][j][3] = 0.f;
    const long long ks = (N + 15) / 16;
    const long long per = (ks + gridDim.x - 1) / gridDim.x;
    const long long k0 = blockIdx.x * per, k1 = min(ks, k0 + per);
    for (long long kk = k0; kk < k1; ++kk) {
        const long long p = kk * 16 + 2 * t;
        auto ld2 = [&](const float* X, int row, int rows, long long q) -> float2 {
            if (row >= rows) return make_float2(0.f, 0.f);
            const float* r = X + (long long)row * N + q;
            return make_float2(q < N ? r[0] : 0.f, q + 1 < N ? r[1] : 0.f);
        };
        unsigned bh[NT][2], bl[NT][2];
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            const float2 v0 = ld2(V, j * 8 + g, B, p), v1 = ld2(V, j * 8 + g, B, p + 8);
            split2(v0.x, v0.y, bh[j][0], bl[j][0]);
            split2(v1.x, v1.y, bh[j][1], bl[j][1]);
        }
#pragma unroll
        for (int i = 0; i < MTW; ++i) {
            const int mt = warp + i * kMmaWarps;
            if (mt >= MT) break;
            const float2 u0 = ld2(U, mt * 16 + g, A, p), u1 = ld2(U, mt * 16 + g + 8, A, p);
            const float2 u2 = ld2(U, mt * 16 + g, A, p + 8), u3 = ld2(U, mt * 16 + g + 8, A, p + 8);
            unsigned ah[4], al[4];
            split2(u0.x, u0.y, ah[0], al[0]);
            split2(u1.x, u1.y, ah[1], al[1]);
            split2(u2.x, u2.y, ah[2], al[2]);
            split2(u3.x, u3.y, ah[3], al[3]);
#pragma unroll
            for (int j = 0; j < NT; ++j) mma3(acc[i][j], ah, al, bh[j][0], bh[j][1], bl[j][0], bl[j][1]);
        }
    }
    const int E = A * B;
#pragma unroll
    for (int i = 0; i < MTW; ++i) {
        const int mt = warp + i * kMmaWarps;
        if (mt >= MT) break;
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int a = mt * 16 + g + ((r & 2) ? 8 : 0), b = j * 8 + 2 * t + (r & 1);
                if (a < A && b < B) part[(long long)blockIdx.x * E + (long long)a * B + b] = acc[i][j][r];
            }
    }
}

inline int grid_for(long long n) {
    long long g = (n + kT - 1) / kT;
    if (g > 152 * 16) g = 152 * 16;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

// ---------------------------------------------------------------------------
// object
// ---------------------------------------------------------------------------
struct pf_fno {
    FnoDims d{};
    int dev = 0;
    cudaStream_t s = nullptr;
    int bf16 = 1;
    long long npar = 0;
    // parameter offsets
    long long oP, op, oQ1, oq1, oQ2, oq2;
    std::vector<long long> oW, oV, ov;
    float *theta = nullptr, *grad = nullptr, *am = nullptr, *av = nullptr;
    __nv_bfloat162* wbf = nullptr;  // BF16 copies of all spectral weights (same layout)
    long long nW = 0;               // complex entries per layer (K C C)
    int adam_t = 0;
    // DFT matrices
    float2 *Mx = nullptr, *Mxw = nullptr, *My = nullptr, *Mz = nullptr;      // forward (Mxw: scaled w/N)
    float2 *IXw = nullptr, *IX1 = nullptr, *IY = nullptr, *IZ = nullptr;     // inverse
    // activations / work
    float *x = nullptr, *act = nullptr, *zs = nullptr, *hpre = nullptr, *hh = nullptr, *out = nullptr;
    float2 *Ak = nullptr;            // A_l per layer [L][C][K]
    float2 *T1 = nullptr, *T2 = nullptr, *Ok = nullptr, *Gk = nullptr;
    float *sbuf = nullptr, *da = nullptr, *dz = nullptr, *dh = nullptr, *dout = nullptr;
    float* part = nullptr;
    int npart_blk = 0;
    double* dpart = nullptr;
    double* hsum = nullptr;  // pinned
    float4 in_mean{0, 0, 0, 0}, in_istd{1, 1, 1, 1}, out_std{1, 1, 1, 1};
    double* realbuf = nullptr;  // real-space FP64 state [4][N]: the proposal
    double* realbuf2 = nullptr; // real-space FP64 state [4][N]: the verified integration
    float* tgt = nullptr;       // training target [4][N]
    char err[256] = "no error";
};

namespace {

thread_local char g_fno_err[256] = "no error";

int ffail(pf_fno* f, int code, const char* msg, cudaError_t e = cudaSuccess) {
    char* dst = f ? f->err : g_fno_err;
    if (e != cudaSuccess)
        std::snprintf(dst, 256, "%s: %s", msg, cudaGetErrorString(e));
    else
        std::snprintf(dst, 256, "%s", msg);
    return code;
}

template <typename P>
cudaError_t falloc(P** p, size_t bytes) {
    cudaError_t e = cudaMalloc((void**)p, bytes);
    if (e != cudaSuccess) cudaGetLastError();
    return e;
}

void fno_free(pf_fno* f) {
    void* ps[] = {f->theta, f->grad, f->am, f->av, f->wbf, f->Mx, f->Mxw, f->My, f->Mz, f->IXw, f->IX1, f->IY,
                  f->IZ, f->x, f->act, f->zs, f->hpre, f->hh, f->out, f->Ak, f->T1, f->T2, f->Ok, f->Gk,
                  f->sbuf, f->da, f->dz, f->dh, f->dout, f->part, f->dpart, f->realbuf, f->realbuf2, f->tgt};
    for (void* p : ps) cudaFree(p);
    if (f->hsum) cudaFreeHost(f->hsum);
}

void axis_launch(cudaStream_t s, bool in_real, bool out_real, bool accum, const void* in, void* out,
                 const float2* M, int nk, int nj, long long n_outer, int n_inner) {
    const size_t sm = (size_t)nk * nj * sizeof(float2);
    const int g = grid_for(n_outer * nk * n_inner);
    if (in_real && !out_real)
        k_axis<true, false, false><<<g, kT, sm, s>>>(in, out, M, nk, nj, n_outer, n_inner);
    else if (!in_real && !out_real)
        k_axis<false, false, false><<<g, kT, sm, s>>>(in, out, M, nk, nj, n_outer, n_inner);
    else if (!accum)
        k_axis<false, true, false><<<g, kT, sm, s>>>(in, out, M, nk, nj, n_outer, n_inner);
    else
        k_axis<false, true, true><<<g, kT, sm, s>>>(in, out, M, nk, nj, n_outer, n_inner);
}

// A = F_K(a): a [C][nz][ny][nx] real -> A [C][2m][2m][m]
void trunc_dft(pf_fno* f, const float* a, float2* A, const float2* Mx) {
    const FnoDims& d = f->d;
    axis_launch(f->s, true, false, false, a, f->T1, Mx, d.m, d.nx, (long long)d.C * d.nz * d.ny, 1);
    axis_launch(f->s, false, false, false, f->T1, f->T2, f->My, 2 * d.m, d.ny, (long long)d.C * d.nz, d.m);
    axis_launch(f->s, false, false, false, f->T2, A, f->Mz, 2 * d.m, d.nz, (long long)d.C, 2 * d.m * d.m);
}

// r (=|+=) Re F^-1 (O) with the x matrix IX (weights and 1/N folded in)
void trunc_inv(pf_fno* f, const float2* O, float* r, const float2* IX, bool accum) {
    const FnoDims& d = f->d;
    axis_launch(f->s, false, false, false, O, f->T2, f->IZ, d.nz, 2 * d.m, (long long)d.C, 2 * d.m * d.m);
    axis_launch(f->s, false, false, false, f->T2, f->T1, f->IY, d.ny, 2 * d.m, (long long)d.C * d.nz, d.m);
    axis_launch(f->s, false, true, accum, f->T1, r, IX, d.nx, d.m, (long long)d.C * d.nz * d.ny, 1);
}

// G[A][B] = sum_p U[a][p] V[b][p] into dst (V null: sums of U rows)
// tensor-core launch of the outer-product reduction (BF16 mode, V present)
template <int MTW, int NT>
void outer_mma_launch(pf_fno* f, const float* U, const float* V, int A, int B) {
    k_outer_mma<MTW, NT><<<f->npart_blk, 32 * kMmaWarps, 0, f->s>>>(U, V, A, B, f->d.N, f->part);
}

bool outer_mma(pf_fno* f, const float* U, const float* V, int A, int B) {
    if (!f->bf16 || !V) return false;
    const int MT = (A + 15) / 16, NT = (B + 7) / 8, MTW = (MT + kMmaWarps - 1) / kMmaWarps;
    // register budget: MTW * NT * 4 accumulators per lane
    if (MTW == 1 && NT == 1) outer_mma_launch<1, 1>(f, U, V, A, B);
    else if (MTW == 1 && NT <= 4) outer_mma_launch<1, 4>(f, U, V, A, B);
    else if (MTW == 1 && NT <= 8) outer_mma_launch<1, 8>(f, U, V, A, B);
    else if (MTW == 1 && NT <= 16) outer_mma_launch<1, 16>(f, U, V, A, B);
    else if (MTW == 2 && NT <= 4) outer_mma_launch<2, 4>(f, U, V, A, B);
    else if (MTW == 2 && NT <= 8) outer_mma_launch<2, 8>(f, U, V, A, B);
    else return false;
    return true;
}

void outer_reduce(pf_fno* f, const float* U, const float* V, int A, int B, float* dst) {
    const int nb = f->npart_blk;
    if (!outer_mma(f, U, V, A, B)) {
        const size_t sm = (size_t)(A + B) * kCh * sizeof(float);
        k_outer_partial<<<nb, kT, sm, f->s>>>(U, V, A, B, f->d.N, f->part);
    }
    k_sum_partials<<<grid_for(A * B), kT, 0, f->s>>>(f->part, nb, A * B, dst);
}

template <int MT, bool TRANS>
void dense_mma_launch(pf_fno* f, const float* x, float* y, float* zout, const float* Mw, const float* b,
                      const float* add, int A, int B, int act, int accum) {
    const int K = TRANS ? A : B, KT = (K + 15) / 16;
    const size_t sm = (size_t)MT * KT * 256 * sizeof(unsigned);
    long long nt = (f->d.N + 7) / 8;
    long long grid = (nt + kMmaWarps - 1) / kMmaWarps;
    if (grid > 152 * 8) grid = 152 * 8;
    auto k = k_dense_mma<MT, TRANS>;
    if (sm > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k<<<(int)grid, 32 * kMmaWarps, sm, f->s>>>(x, y, zout, Mw, b, add, A, B, f->d.N, act, accum);
}

template <bool TRANS>
bool dense_mma(pf_fno* f, const float* x, float* y, float* zout, const float* Mw, const float* b, const float* add,
               int A, int B, int act, int accum) {
    if (!f->bf16) return false;
    const int M = TRANS ? B : A;
    switch ((M + 15) / 16) {
        case 1: dense_mma_launch<1, TRANS>(f, x, y, zout, Mw, b, add, A, B, act, accum); return true;
        case 2: dense_mma_launch<2, TRANS>(f, x, y, zout, Mw, b, add, A, B, act, accum); return true;
        case 4: dense_mma_launch<4, TRANS>(f, x, y, zout, Mw, b, add, A, B, act, accum); return true;
        case 8: dense_mma_launch<8, TRANS>(f, x, y, zout, Mw, b, add, A, B, act, accum); return true;
        default: return false;
    }
}

void dense(pf_fno* f, const float* x, float* y, float* zout, const float* Mw, const float* b, const float* add, int A,
           int B, int act) {
    if (dense_mma<false>(f, x, y, zout, Mw, b, add, A, B, act, 0)) return;
    const size_t sm = (size_t)(A * B + A) * sizeof(float);
    k_dense<<<grid_for(f->d.N), kT, sm, f->s>>>(x, y, zout, Mw, b, add, A, B, f->d.N, act);
}

void dense_t(pf_fno* f, const float* dy, float* dx, const float* Mw, int A, int B, int accum) {
    if (dense_mma<true>(f, dy, dx, nullptr, Mw, nullptr, nullptr, A, B, 0, accum)) return;
    const size_t sm = (size_t)(A * B) * sizeof(float);
    k_dense_t<<<grid_for(f->d.N), kT, sm, f->s>>>(dy, dx, Mw, A, B, f->d.N, accum);
}

int fno_forward(pf_fno* f, const float* x) {
    const FnoDims& d = f->d;
    const long long N = d.N;
    cudaStream_t s = f->s;
    if (x != f->x) cudaMemcpyAsync(f->x, x, sizeof(float) * 4 * N, cudaMemcpyDeviceToDevice, s);
    float* a0 = f->act;
    dense(f, f->x, a0, nullptr, f->theta + f->oP, f->theta + f->op, nullptr, d.C, d.cin, 0);
    for (int l = 0; l < d.L; ++l) {
        float* a = f->act + (size_t)l * d.C * N;
        float* an = f->act + (size_t)(l + 1) * d.C * N;
        float2* A = f->Ak + (size_t)l * d.C * d.K;
        trunc_dft(f, a, A, f->Mx);
        const float2* w32 = reinterpret_cast<const float2*>(f->theta + f->oW[l]);
        const __nv_bfloat162* w16 = f->bf16 ? f->wbf + (size_t)l * f->nW : nullptr;
        k_mix<<<grid_for((long long)d.C * d.K), kT, 0, s>>>(A, f->Ok, w32, w16, d.C, d.K);
        trunc_inv(f, f->Ok, f->sbuf, f->IXw, false);
        dense(f, a, an, f->zs + (size_t)l * d.C * N, f->theta + f->oV[l], f->theta + f->ov[l], f->sbuf, d.C, d.C,
              l < d.L - 1 ? 1 : 0);
    }
    float* aL = f->act + (size_t)d.L * d.C * N;
    dense(f, aL, f->hh, f->hpre, f->theta + f->oQ1, f->theta + f->oq1, nullptr, d.H, d.C, 1);
    dense(f, f->hh, f->out, nullptr, f->theta + f->oQ2, f->theta + f->oq2, nullptr, d.cin, d.H, 0);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PF_OK : ffail(f, PF_ECUDA, "fno forward", e);
}

int fno_backward(pf_fno* f, const float* tgt, double* loss) {
    const FnoDims& d = f->d;
    const long long N = d.N;
    cudaStream_t s = f->s;
    const int nb = 152 * 4;
    k_mse<<<nb, kT, 0, s>>>(f->out, tgt, f->dout, 4 * N, f->dpart);
    float* G = f->grad;
    outer_reduce(f, f->dout, f->hh, d.cin, d.H, G + f->oQ2);
    outer_reduce(f, f->dout, nullptr, d.cin, 1, G + f->oq2);
    dense_t(f, f->dout, f->dh, f->theta + f->oQ2, d.cin, d.H, 0);
    k_gelu_bwd<<<grid_for((long long)d.H * N), kT, 0, s>>>(f->dh, f->hpre, (long long)d.H * N);
    float* aL = f->act + (size_t)d.L * d.C * N;
    outer_reduce(f, f->dh, aL, d.H, d.C, G + f->oQ1);
    outer_reduce(f, f->dh, nullptr, d.H, 1, G + f->oq1);
    dense_t(f, f->dh, f->da, f->theta + f->oQ1, d.H, d.C, 0);
    for (int l = d.L - 1; l >= 0; --l) {
        float* a = f->act + (size_t)l * d.C * N;
        float* z = f->zs + (size_t)l * d.C * N;
        cudaMemcpyAsync(f->dz, f->da, sizeof(float) * d.C * N, cudaMemcpyDeviceToDevice, s);
        if (l < d.L - 1) k_gelu_bwd<<<grid_for((long long)d.C * N), kT, 0, s>>>(f->dz, z, (long long)d.C * N);
        outer_reduce(f, f->dz, a, d.C, d.C, G + f->oV[l]);
        outer_reduce(f, f->dz, nullptr, d.C, 1, G + f->ov[l]);
        dense_t(f, f->dz, f->da, f->theta + f->oV[l], d.C, d.C, 0);
        // spectral: GO = (w/N) F(dz); GW, GA; da += Re F^-1 (GA) (unweighted)
        trunc_dft(f, f->dz, f->Gk, f->Mxw);
        const float2* w32 = reinterpret_cast<const float2*>(f->theta + f->oW[l]);
        const __nv_bfloat162* w16 = f->bf16 ? f->wbf + (size_t)l * f->nW : nullptr;
        float2* A = f->Ak + (size_t)l * d.C * d.K;
        k_mix_bwd<<<grid_for((long long)d.C * d.K), kT, 0, s>>>(f->Gk, A, f->Ok, reinterpret_cast<float2*>(G + f->oW[l]),
                                                                w32, w16, d.C, d.K);
        trunc_inv(f, f->Ok, f->da, f->IX1, true);
    }
    outer_reduce(f, f->da, f->x, d.C, d.cin, G + f->oP);
    outer_reduce(f, f->da, nullptr, d.C, 1, G + f->op);
    if (loss) {
        double* tot = f->dpart + nb;
        launch_reduce(f->dpart, nb, 1.0 / (4.0 * (double)N), tot, s);
        cudaMemcpyAsync(f->hsum, tot, sizeof(double), cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return ffail(f, PF_ECUDA, "fno backward", e);
        *loss = f->hsum[0];
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PF_OK : ffail(f, PF_ECUDA, "fno backward", e);
}

void refresh_bf16(pf_fno* f) {
    for (int l = 0; l < f->d.L; ++l)
        k_to_bf16<<<grid_for(f->nW), kT, 0, f->s>>>(reinterpret_cast<const float2*>(f->theta + f->oW[l]),
                                                   f->wbf + (size_t)l * f->nW, f->nW);
}

void build_matrices(pf_fno* f, std::vector<float2>& Mx, std::vector<float2>& Mxw, std::vector<float2>& My,
                    std::vector<float2>& Mz, std::vector<float2>& IXw, std::vector<float2>& IX1,
                    std::vector<float2>& IY, std::vector<float2>& IZ) {
    const FnoDims& d = f->d;
    const double tp = 6.283185307179586476925286766559;
    auto kidx = [&](int n, int j) { return j < d.m ? j : n - 2 * d.m + j; };
    Mx.resize((size_t)d.m * d.nx);
    Mxw.resize(Mx.size());
    IXw.resize((size_t)d.nx * d.m);
    IX1.resize(IXw.size());
    for (int k = 0; k < d.m; ++k)
        for (int x = 0; x < d.nx; ++x) {
            const double th = tp * (double)((long long)k * x % d.nx) / d.nx;
            const double c = std::cos(th), sn = std::sin(th), w = (k == 0 ? 1.0 : 2.0);
            Mx[(size_t)k * d.nx + x] = make_float2((float)c, (float)-sn);
            Mxw[(size_t)k * d.nx + x] = make_float2((float)(c * w / d.N), (float)(-sn * w / d.N));
            IXw[(size_t)x * d.m + k] = make_float2((float)(c * w / d.N), (float)(sn * w / d.N));
            IX1[(size_t)x * d.m + k] = make_float2((float)c, (float)sn);
        }
    auto axis = [&](int n, std::vector<float2>& F, std::vector<float2>& I) {
        F.resize((size_t)2 * d.m * n);
        I.resize(F.size());
        for (int j = 0; j < 2 * d.m; ++j) {
            const int k = kidx(n, j);
            for (int x = 0; x < n; ++x) {
                const double th = tp * (double)((long long)k * x % n) / n;
                F[(size_t)j * n + x] = make_float2((float)std::cos(th), (float)-std::sin(th));
                I[(size_t)x * 2 * d.m + j] = make_float2((float)std::cos(th), (float)std::sin(th));
            }
        }
    };
    axis(d.ny, My, IY);
    axis(d.nz, Mz, IZ);
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

int pf_fno_create(int nx, int ny, int nz, int C, int modes, int H, int L, int bf16, void* cuda_stream, pf_fno** out) {
    if (!out) return ffail(nullptr, PF_EINVAL, "pf_fno_create: NULL out");
    *out = nullptr;
    if (nx < 4 || ny < 4 || nz < 4 || C < 1 || C > 64 || H < 1 || H > 256 || L < 1 || L > 8 || modes < 1 ||
        2 * modes > ny || 2 * modes > nz || modes > nx / 2 || C * H > 4096 || C * C > 4096)
        return ffail(nullptr, PF_EINVAL, "pf_fno_create: unsupported dimensions");
    pf_fno* f = new (std::nothrow) pf_fno();
    if (!f) return ffail(nullptr, PF_ENOMEM, "host allocation failed");
    cudaGetDevice(&f->dev);
    f->s = (cudaStream_t)cuda_stream;
    f->bf16 = bf16 ? 1 : 0;
    FnoDims& d = f->d;
    d.nx = nx;
    d.ny = ny;
    d.nz = nz;
    d.C = C;
    d.m = modes;
    d.H = H;
    d.L = L;
    d.cin = 4;
    d.N = (long long)nx * ny * nz;
    d.K = 4 * modes * modes * modes;
    f->nW = (long long)d.K * C * C;
    long long o = 0;
    f->oP = o;
    o += (long long)C * d.cin;
    f->op = o;
    o += C;
    for (int l = 0; l < L; ++l) {
        f->oW.push_back(o);
        o += 2 * f->nW;
        f->oV.push_back(o);
        o += (long long)C * C;
        f->ov.push_back(o);
        o += C;
    }
    f->oQ1 = o;
    o += (long long)H * C;
    f->oq1 = o;
    o += H;
    f->oQ2 = o;
    o += (long long)d.cin * H;
    f->oq2 = o;
    o += d.cin;
    f->npar = o;
    const long long N = d.N;
    f->npart_blk = 152 * 4;
    cudaError_t e = cudaSuccess;
    auto A = [&](auto** p, size_t bytes) {
        if (e == cudaSuccess) e = falloc(p, bytes);
    };
    A(&f->theta, sizeof(float) * f->npar);
    A(&f->grad, sizeof(float) * f->npar);
    A(&f->am, sizeof(float) * f->npar);
    A(&f->av, sizeof(float) * f->npar);
    A(&f->wbf, sizeof(__nv_bfloat162) * f->nW * L);
    A(&f->x, sizeof(float) * 4 * N);
    A(&f->act, sizeof(float) * (size_t)(L + 1) * C * N);
    A(&f->zs, sizeof(float) * (size_t)L * C * N);
    A(&f->hpre, sizeof(float) * (size_t)H * N);
    A(&f->hh, sizeof(float) * (size_t)H * N);
    A(&f->out, sizeof(float) * 4 * N);
    A(&f->Ak, sizeof(float2) * (size_t)L * C * d.K);
    A(&f->T1, sizeof(float2) * (size_t)C * nz * ny * modes);
    A(&f->T2, sizeof(float2) * (size_t)C * nz * 2 * modes * modes);
    A(&f->Ok, sizeof(float2) * (size_t)C * d.K);
    A(&f->Gk, sizeof(float2) * (size_t)C * d.K);
    A(&f->sbuf, sizeof(float) * (size_t)C * N);
    A(&f->da, sizeof(float) * (size_t)C * N);
    A(&f->dz, sizeof(float) * (size_t)C * N);
    A(&f->dh, sizeof(float) * (size_t)H * N);
    A(&f->dout, sizeof(float) * 4 * N);
    A(&f->tgt, sizeof(float) * 4 * N);
    A(&f->part, sizeof(float) * (size_t)f->npart_blk * (size_t)(H * C > C * C ? H * C : C * C));
    A(&f->dpart, sizeof(double) * (152 * 4 * 16 + 32));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&f->hsum, sizeof(double) * 2);
    std::vector<float2> Mx, Mxw, My, Mz, IXw, IX1, IY, IZ;
    build_matrices(f, Mx, Mxw, My, Mz, IXw, IX1, IY, IZ);
    A(&f->Mx, Mx.size() * sizeof(float2));
    A(&f->Mxw, Mxw.size() * sizeof(float2));
    A(&f->My, My.size() * sizeof(float2));
    A(&f->Mz, Mz.size() * sizeof(float2));
    A(&f->IXw, IXw.size() * sizeof(float2));
    A(&f->IX1, IX1.size() * sizeof(float2));
    A(&f->IY, IY.size() * sizeof(float2));
    A(&f->IZ, IZ.size() * sizeof(float2));
    if (e == cudaSuccess) {
        struct {
            float2* d;
            std::vector<float2>* h;
        } cp[] = {{f->Mx, &Mx}, {f->Mxw, &Mxw}, {f->My, &My}, {f->Mz, &Mz},
                  {f->IXw, &IXw}, {f->IX1, &IX1}, {f->IY, &IY}, {f->IZ, &IZ}};
        for (auto& c : cp)
            if (e == cudaSuccess) e = cudaMemcpy(c.d, c.h->data(), c.h->size() * sizeof(float2), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemset(f->am, 0, sizeof(float) * f->npar);
    if (e == cudaSuccess) e = cudaMemset(f->av, 0, sizeof(float) * f->npar);
    if (e == cudaSuccess) e = cudaMemset(f->theta, 0, sizeof(float) * f->npar);
    if (e != cudaSuccess) {
        ffail(nullptr, e == cudaErrorMemoryAllocation ? PF_ENOMEM : PF_ECUDA, "pf_fno_create", e);
        fno_free(f);
        delete f;
        return e == cudaErrorMemoryAllocation ? PF_ENOMEM : PF_ECUDA;
    }
    *out = f;
    return PF_OK;
}

void pf_fno_destroy(pf_fno* f) {
    if (!f) return;
    cudaSetDevice(f->dev);
    cudaStreamSynchronize(f->s);
    fno_free(f);
    delete f;
}

long long pf_fno_num_params(const pf_fno* f) { return f ? f->npar : -1; }

int pf_fno_set_params(pf_fno* f, const float* theta, long long n) {
    if (!f || !theta || n != f->npar) return ffail(f, PF_EINVAL, "pf_fno_set_params: bad argument");
    cudaSetDevice(f->dev);
    cudaError_t e = cudaMemcpyAsync(f->theta, theta, sizeof(float) * n, cudaMemcpyHostToDevice, f->s);
    if (e == cudaSuccess) {
        refresh_bf16(f);
        e = cudaStreamSynchronize(f->s);
    }
    f->adam_t = 0;
    if (e == cudaSuccess) e = cudaMemsetAsync(f->am, 0, sizeof(float) * n, f->s);
    if (e == cudaSuccess) e = cudaMemsetAsync(f->av, 0, sizeof(float) * n, f->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(f->s);
    return e == cudaSuccess ? PF_OK : ffail(f, PF_ECUDA, "pf_fno_set_params", e);
}

int pf_fno_get_params(pf_fno* f, float* theta, long long n) {
    if (!f || !theta || n != f->npar) return ffail(f, PF_EINVAL, "pf_fno_get_params: bad argument");
    cudaSetDevice(f->dev);
    cudaError_t e = cudaMemcpyAsync(theta, f->theta, sizeof(float) * n, cudaMemcpyDeviceToHost, f->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(f->s);
    return e == cudaSuccess ? PF_OK : ffail(f, PF_ECUDA, "pf_fno_get_params", e);
}

int pf_fno_get_grads(pf_fno* f, float* g, long long n) {
    if (!f || !g || n != f->npar) return ffail(f, PF_EINVAL, "pf_fno_get_grads: bad argument");
    cudaSetDevice(f->dev);
    cudaError_t e = cudaMemcpyAsync(g, f->grad, sizeof(float) * n, cudaMemcpyDeviceToHost, f->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(f->s);
    return e == cudaSuccess ? PF_OK : ffail(f, PF_ECUDA, "pf_fno_get_grads", e);
}

int pf_fno_set_norm(pf_fno* f, const float* in_mean, const float* in_std, const float* out_std) {
    if (!f || !in_mean || !in_std || !out_std) return ffail(f, PF_EINVAL, "pf_fno_set_norm: NULL argument");
    f->in_mean = make_float4(in_mean[0], in_mean[1], in_mean[2], in_mean[3]);
    f->in_istd = make_float4(1.f / in_std[0], 1.f / in_std[1], 1.f / in_std[2], 1.f / in_std[3]);
    f->out_std = make_float4(out_std[0], out_std[1], out_std[2], out_std[3]);
    return PF_OK;
}

int pf_fno_forward(pf_fno* f, const float* x_dev, float* out_dev) {
    if (!f || !x_dev) return ffail(f, PF_EINVAL, "pf_fno_forward: NULL argument");
    cudaSetDevice(f->dev);
    int rc = fno_forward(f, x_dev);
    if (rc) return rc;
    if (out_dev)
        cudaMemcpyAsync(out_dev, f->out, sizeof(float) * 4 * f->d.N, cudaMemcpyDeviceToDevice, f->s);
    cudaError_t e = cudaStreamSynchronize(f->s);
    return e == cudaSuccess ? PF_OK : ffail(f, PF_ECUDA, "pf_fno_forward", e);
}

int pf_fno_backward(pf_fno* f, const float* target_dev, double* loss_out) {
    if (!f || !target_dev) return ffail(f, PF_EINVAL, "pf_fno_backward: NULL argument");
    cudaSetDevice(f->dev);
    double l = 0.0;
    int rc = fno_backward(f, target_dev, &l);
    if (loss_out) *loss_out = l;
    return rc;
}

int pf_fno_adam(pf_fno* f, float lr, float b1, float b2, float eps) {
    if (!f) return ffail(f, PF_EINVAL, "pf_fno_adam: NULL argument");
    cudaSetDevice(f->dev);
    f->adam_t += 1;
    const float c1 = 1.f - powf(b1, (float)f->adam_t), c2 = 1.f - powf(b2, (float)f->adam_t);
    k_adam<<<grid_for(f->npar), kT, 0, f->s>>>(f->theta, f->grad, f->am, f->av, f->npar, lr, b1, b2, eps, c1, c2);
    refresh_bf16(f);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PF_OK : ffail(f, PF_ECUDA, "pf_fno_adam", e);
}

int pf_fno_train_step(pf_fno* f, const float* x_dev, const float* target_dev, float lr, double* loss_out) {
    if (!f || !x_dev || !target_dev) return ffail(f, PF_EINVAL, "pf_fno_train_step: NULL argument");
    cudaSetDevice(f->dev);
    int rc = fno_forward(f, x_dev);
    if (!rc) rc = pf_fno_backward(f, target_dev, loss_out);
    if (!rc) rc = pf_fno_adam(f, lr, 0.9f, 0.999f, 1e-8f);
    return rc;
}

const char* pf_fno_last_error(const pf_fno* f) { return f ? f->err : g_fno_err; }

// Normalisation statistics from solver snapshots (device FP32
// [n_traj][n_snap][4][N]): per-channel mean and standard deviation of the
// inputs and standard deviation of the increments over consecutive pairs.
int pf_fno_fit_norm(pf_fno* f, const float* snaps_dev, int n_traj, int n_snap) {
    if (!f || !snaps_dev || n_traj < 1 || n_snap < 2) return ffail(f, PF_EINVAL, "pf_fno_fit_norm: bad argument");
    cudaSetDevice(f->dev);
    const int nb = 152 * 4;
    k_pair_stats<<<nb, kT, 0, f->s>>>(snaps_dev, n_traj, n_snap, f->d.N, f->dpart);
    std::vector<double> part((size_t)nb * 16);
    cudaError_t e = cudaMemcpyAsync(part.data(), f->dpart, sizeof(double) * part.size(), cudaMemcpyDeviceToHost, f->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(f->s);
    if (e != cudaSuccess) return ffail(f, PF_ECUDA, "pf_fno_fit_norm", e);
    double sum[16] = {};
    for (int b = 0; b < nb; ++b)
        for (int q = 0; q < 16; ++q) sum[q] += part[(size_t)b * 16 + q];
    const double cnt = (double)n_traj * (n_snap - 1) * (double)f->d.N;
    float mean[4], sd[4], dsd[4];
    for (int c = 0; c < 4; ++c) {
        const double m = sum[4 * c] / cnt, v = sum[4 * c + 1] / cnt - m * m;
        const double dm = sum[4 * c + 2] / cnt, dv = sum[4 * c + 3] / cnt - dm * dm;
        mean[c] = (float)m;
        sd[c] = (float)std::fmax(std::sqrt(std::fmax(v, 0.0)), 1e-6);
        dsd[c] = (float)std::fmax(std::sqrt(std::fmax(dv, 0.0)), 1e-9);
    }
    return pf_fno_set_norm(f, mean, sd, dsd);
}

// One Adam step on the pair (s_t, s_{t+tau}) (device FP32 [4][N] each): the
// normalised input and increment target are formed on the device.
int pf_fno_train_pair(pf_fno* f, const float* s0_dev, const float* s1_dev, float lr, double* loss_out) {
    if (!f || !s0_dev || !s1_dev) return ffail(f, PF_EINVAL, "pf_fno_train_pair: NULL argument");
    cudaSetDevice(f->dev);
    const float4 io = make_float4(1.f / f->out_std.x, 1.f / f->out_std.y, 1.f / f->out_std.z, 1.f / f->out_std.w);
    k_pair_prep<<<grid_for(4 * f->d.N), kT, 0, f->s>>>(s0_dev, s1_dev, f->x, f->tgt, f->d.N, f->in_mean, f->in_istd,
                                                      io);
    int rc = fno_forward(f, f->x);
    if (!rc) rc = pf_fno_backward(f, f->tgt, loss_out);
    if (!rc) rc = pf_fno_adam(f, lr, 0.9f, 0.999f, 1e-8f);
    return rc;
}

// Surrogate proposal judged by the integrator (one call = one proposal over
// tau): the network proposes y(t + tau) from y(t); the context then
// integrates the same interval with its adaptive controller (first step h),
// and the proposal is reported as accepted when its WRMS distance to that
// verified integration is <= 1.  The context ends at the verified state.
int pf_surrogate_step(pf_ctx* ctx, pf_fno* f, double tau, double h, double rtol, double atol, int* accepted,
                      double* dist) {
    if (!ctx || !f || !accepted || !(tau > 0) || !(h > 0) || !(rtol >= 0) || !(atol > 0))
        return ffail(f, PF_EINVAL, "pf_surrogate_step: bad argument");
    pf_grid g{};
    double t0 = 0, h0 = 0;
    pf_get_time(ctx, &t0, &h0);
    cudaSetDevice(f->dev);
    int rc = pf_ctx_grid(ctx, &g);
    if (rc) return rc;
    if (g.nx != f->d.nx || g.ny != f->d.ny || g.nz != f->d.nz)
        return ffail(f, PF_EINVAL, "pf_surrogate_step: network and simulation grids differ");
    const long long N = f->d.N;
    cudaError_t e = cudaSuccess;
    if (!f->realbuf) {
        e = falloc(&f->realbuf, sizeof(double) * 4 * N);
        if (e == cudaSuccess) e = falloc(&f->realbuf2, sizeof(double) * 4 * N);
        if (e != cudaSuccess) return ffail(f, PF_ENOMEM, "pf_surrogate_step: allocation", e);
    }
    // proposal y^(t + tau) = y(t) + net(y(t)) in real space (FP64)
    rc = pf_get_state(ctx, f->realbuf, 1);
    if (rc) return rc;
    k_norm_in<<<grid_for(4 * N), kT, 0, f->s>>>(f->realbuf, f->x, N, f->in_mean, f->in_istd);
    rc = fno_forward(f, f->x);
    if (rc) return rc;
    k_apply_delta<<<grid_for(4 * N), kT, 0, f->s>>>(f->realbuf, f->out, N, f->out_std);
    e = cudaStreamSynchronize(f->s);
    if (e != cudaSuccess) return ffail(f, PF_ECUDA, "pf_surrogate_step: proposal", e);
    // the verified integration of the same interval
    pf_set_time(ctx, t0, h);
    pf_stats st{};
    rc = pf_advance(ctx, t0 + tau, rtol, atol, &st);
    if (rc) return rc;
    rc = pf_get_state(ctx, f->realbuf2, 1);
    if (rc) return rc;
    const int nb = 152 * 4;
    k_wrms_dist<<<nb, kT, 0, f->s>>>(f->realbuf, f->realbuf2, 4 * N, rtol, atol, f->dpart);
    double* tot = f->dpart + nb;
    launch_reduce(f->dpart, nb, 1.0 / (4.0 * (double)N), tot, f->s);
    e = cudaMemcpyAsync(f->hsum, tot, sizeof(double), cudaMemcpyDeviceToHost, f->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(f->s);
    if (e != cudaSuccess) return ffail(f, PF_ECUDA, "pf_surrogate_step: distance", e);
    const double d = std::sqrt(f->hsum[0]);
    if (dist) *dist = d;
    *accepted = (std::isfinite(d) && d <= 1.0) ? 1 : 0;
    return PF_OK;
}

}  // extern "C"
