// x passes: packed real transforms along the contiguous axis with the
// real-space physics of the right-hand side, the WRMS error norm and the
// real-space free energy fused in.
#pragma once
#include "pf_common.cuh"

namespace pf {
// ---------------------------------------------------------------------------
// x passes: packed real transforms with the real-space physics fused in.
// Two consecutive rows (y, y+1) of one field share one complex line
// z = a + i b; C2R packs Z_k = A_k + i B_k (Hermitian extension for k > n/2,
// imaginary parts of DC and Nyquist dropped), R2C unpacks
// A_k = (Z_k + conj Z_{n-k})/2, B_k = (Z_k - conj Z_{n-k})/(2i).
// ---------------------------------------------------------------------------
// a / b: the FP32 form divides through the hardware reciprocal (about two
// ulp, far inside the FP32 transforms' rounding); FP64 divides exactly
template <typename T>
__device__ __forceinline__ T xdiv(T a, T b) {
    if constexpr (sizeof(T) == 4)
        return __fdividef(a, b);
    else
        return a / b;
}

struct Pt {
    // real-space physics at one point (Sec. 4.1); returns q and g_v.  OBST:
    // the literal obstacle barrier instead of the double well (a compile-time
    // choice, so that the default path carries none of its instructions)
    template <typename T, bool OBST = false>
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
        const T mu = xdiv<T>(X - H * Bv - ((T)1 - H) * Bm, denom);
        const T Xm = mu * pt.inv2Am + Bm;
        const T Xv = mu * pt.inv2Av + Bv;
        const T fm = pt.A0m + pt.Am * (Xm - Bm) * (Xm - Bm);
        const T fv = pt.A0v + pt.Av * (Xv - Bv) * (Xv - Bv);
        const T drive = fv - fm - mu * (Xv - Xm);
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            const T f = p[v];
            T d;
            if constexpr (OBST)
                d = pt.wb * ((T)1 - (T)2 * (p[0] + p[1] + p[2]));  // d/dphi_v of omega_bar S (1 - S)
            else
                d = pt.wb2 * f * ((T)1 - f) * ((T)1 - (T)2 * f);
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

// line length nx and half-spectrum length nx/2+1 along x, compile-time when
// NX > 0, and the divisions by them
template <int NX>
struct XLen {
    int n, h;
    unsigned mn, mh;
    __device__ __forceinline__ explicit XLen(const Geo& g)
        : n(NX > 0 ? NX : g.nx), h(NX > 0 ? NX / 2 + 1 : g.nxh), mn(g.mul_nx), mh(g.mul_nxh) {}
    __device__ __forceinline__ int divn(int e) const {
        if constexpr (NX > 0)
            return e / NX;
        else
            return (int)FastDiv((unsigned)n, mn).div((unsigned)e);
    }
    __device__ __forceinline__ int divh(int e) const {
        if constexpr (NX > 0)
            return e / (NX / 2 + 1);
        else
            return (int)FastDiv((unsigned)h, mh).div((unsigned)e);
    }
};

// transform of nl skewed x lines: compile-time plan, or the generic stages
template <int SIGN, int PID, bool R16, typename T2>
__device__ __forceinline__ T2* x_fft(T2* a, T2* b, const AxisPlan& p, int nl, int ls) {
    if constexpr (PID > 0)
        return fft_fixed_run<SIGN, FixedPlan<PID>::N, 1>(a, b, nl, ls, twiddles<T2>(p), typename FixedPlan<PID>::Rad{});
    else
        return fft_lines<SIGN, false, 0, true, R16>(a, b, p, nl, 1, ls);
}

// load F packed lines (C2R input) of row pairs [rp0, rp0+P) into S: the raw
// half-spectrum rows are first copied asynchronously into `raw` (all of a
// tile's loads in flight together), then packed from shared memory
template <int NX, typename T2>
__device__ __forceinline__ void c2r_load_async(const Geo& g, const T2* __restrict__ in, int F, int P, int rp0,
                                               int npairs, T2* S, int ls, T2* raw) {
    const XLen<NX> L(g);
    const int nx = L.n, nh = nx / 2, nxh = L.h;
    for (int e = threadIdx.x; e < P * F * 2 * nxh; e += blockDim.x) {
        const int r = L.divh(e), k = e - r * nxh;  // raw row r = (rp F + f) 2 + (0: row y, 1: row y+1)
        const int pf = r >> 1, rp = F == 4 ? pf >> 2 : pf / 3, f = pf - rp * F;
        if (rp0 + rp < npairs)
            cp_async<sizeof(T2)>(raw + e, in + (long long)f * g.NK + (2LL * (rp0 + rp) + (r & 1)) * nxh + k);
    }
    cp_async_wait_all();
    __syncthreads();
    for (int e = threadIdx.x; e < P * F * nx; e += blockDim.x) {
        const int line = L.divn(e), x = e - line * nx, rp = F == 4 ? line >> 2 : line / 3;
        T2 Z = T2{0, 0};
        if (rp0 + rp < npairs) {
            const int k = x <= nh ? x : nx - x;
            T2 a = raw[(2 * line) * nxh + k], b = raw[(2 * line + 1) * nxh + k];
            if (k == 0 || k == nh) {
                a.y = 0;
                b.y = 0;
            }
            Z = x <= nh ? T2{a.x - b.y, a.y + b.x} : T2{a.x + b.y, b.x - a.y};
        }
        S[line * ls + skew<true>(x)] = Z;
    }
}

// load F packed lines (C2R input) of row pairs [rp0, rp0+P) into S
template <int NX, typename T2>
__device__ __forceinline__ void c2r_load(const Geo& g, const T2* __restrict__ in, int F, int P, int rp0, int npairs,
                                         T2* S, int ls) {
    const XLen<NX> L(g);
    const int nx = L.n, nh = nx / 2, nxh = L.h;
    // unrolled so that several iterations' loads are in flight together
#pragma unroll 4
    for (int e = threadIdx.x; e < P * F * nx; e += blockDim.x) {
        const int line = L.divn(e), x = e - line * nx, rp = F == 4 ? line >> 2 : line / 3, f = line - rp * F;
        T2 Z = T2{0, 0};
        if (rp0 + rp < npairs) {
            const long long row = 2LL * (rp0 + rp);
            const int k = x <= nh ? x : nx - x;
            const T2* base = in + (long long)f * g.NK + row * nxh + k;
            T2 a = base[0], b = base[nxh];
            if (k == 0 || k == nh) {
                a.y = 0;
                b.y = 0;
            }
            if (x <= nh)
                Z = T2{a.x - b.y, a.y + b.x};
            else
                Z = T2{a.x + b.y, b.x - a.y};
        }
        S[line * ls + skew<true>(x)] = Z;
    }
}

template <int NX, typename T2>
__device__ __forceinline__ void r2c_store(const Geo& g, const T2* S, int ls, int F, int P, int rp0, int npairs,
                                          T2* __restrict__ out) {
    using T = decltype(T2{}.x);
    const XLen<NX> L(g);
    const int nx = L.n, nxh = L.h;
    for (int e = threadIdx.x; e < P * F * nxh; e += blockDim.x) {
        const int line = L.divh(e), k = e - line * nxh, rp = F == 4 ? line >> 2 : line / 3, f = line - rp * F;
        if (rp0 + rp >= npairs) continue;
        const T2 Zk = S[line * ls + skew<true>(k)];
        const T2 Zm = S[line * ls + skew<true>(k == 0 ? 0 : nx - k)];
        const T half = (T)0.5;
        const T2 A = T2{(Zk.x + Zm.x) * half, (Zk.y - Zm.y) * half};
        const T2 B = T2{(Zk.y + Zm.y) * half, (Zm.x - Zk.x) * half};
        const long long row = 2LL * (rp0 + rp);
        T2* base = out + (long long)f * g.NK + row * nxh + k;
        base[0] = A;
        base[nxh] = B;
    }
}

template <typename T, bool R16, int PID>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 4 : 3) k_x_pass(Geo g, Phys ph, int mode, const typename Cx<T>::t* __restrict__ in,
                                                     typename Cx<T>::t* __restrict__ out, T* __restrict__ R,
                                                     const T* __restrict__ Rin, double* __restrict__ partials,
                                                     double rtol, double atol, const double* __restrict__ real_in,
                                                     double* __restrict__ real_out, int P) {
    PF_SKIP_INACTIVE(g);
    using T2 = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smraw[];
    constexpr int NX = FixedPlan<PID>::N;
    const XLen<NX> L(g);
    const int nx = L.n;
    const int ls = skewed_len(nx);
    const PhysT<T>& pt = phys_t<T>(ph);
    const int npairs = g.nz * g.ny / 2;
    const int rp0 = blockIdx.x * P;
    T2* S0 = reinterpret_cast<T2*>(smraw);
    T2* S1 = S0 + 4 * P * ls;
    __shared__ double red[kThreads / 32];

    // ---- input: C2R of the incoming half-spectrum lines, or packed real rows
    int Fin = 0;
    if (mode == XM_PHYS1 || mode == XM_WRMS || mode == XM_C2R_REAL || mode == XM_ENERGY) Fin = 4;
    if (mode == XM_PHYS2) Fin = ph.elastic ? 3 : 0;
    const T* Ereal = mode == XM_PHYS2R ? reinterpret_cast<const T*>(in) : nullptr;
    T2* RS = S0;  // real-space lines (a + i b)
    if (mode == XM_R2C_REAL) {
#pragma unroll 4
        for (int e = threadIdx.x; e < P * 4 * nx; e += blockDim.x) {
            const int line = L.divn(e), x = e - line * nx, rp = line >> 2, f = line & 3;
            T2 Z = T2{0, 0};
            if (rp0 + rp < npairs) {
                const long long row = 2LL * (rp0 + rp);
                const double* b = real_in + (long long)f * g.N + row * nx + x;
                Z = T2{(T)b[0], (T)b[nx]};
            }
            S0[line * ls + skew<true>(x)] = Z;
        }
        __syncthreads();
        T2* res = x_fft<-1, PID, R16>(S0, S1, g.px, 4 * P, ls);
        r2c_store<NX>(g, res, ls, 4, P, rp0, npairs, out);
        return;
    }
    if (Fin > 0) {
        // the raw rows of the F fields fit in the second buffer (F (nx + 2) <= 4 ls) for every nx >= 32
        if ((long long)Fin * 2 * L.h <= 4LL * ls)
            c2r_load_async<NX>(g, in, Fin, P, rp0, npairs, S0, ls, S1);
        else
            c2r_load<NX>(g, in, Fin, P, rp0, npairs, S0, ls);
        __syncthreads();
        RS = x_fft<+1, PID, R16>(S0, S1, g.px, Fin * P, ls);
    }
    T2* OS = (RS == S0) ? S1 : S0;  // output lines

    if (mode == XM_C2R_REAL) {
        for (int e = threadIdx.x; e < P * 4 * nx; e += blockDim.x) {
            const int line = L.divn(e), x = e - line * nx, rp = line >> 2, f = line & 3;
            if (rp0 + rp >= npairs) continue;
            const long long row = 2LL * (rp0 + rp);
            const T2 z = RS[line * ls + skew<true>(x)];
            double* b = real_out + (long long)f * g.N + row * nx + x;
            b[0] = (double)z.x;
            b[nx] = (double)z.y;
        }
        return;
    }

    if (mode == XM_WRMS) {
        double acc = 0.0;
        for (int e = threadIdx.x; e < P * 4 * nx; e += blockDim.x) {
            const int line = L.divn(e), x = e - line * nx, rp = line >> 2, f = line & 3;
            if (rp0 + rp >= npairs) continue;
            const long long row = 2LL * (rp0 + rp);
            const T2 z = RS[line * ls + skew<true>(x)];
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
    const bool full_rhs = (mode == XM_PHYS2) || (mode == XM_PHYS2R) || (mode == XM_PHYS1 && !ph.elastic);
#pragma unroll 2
    for (int e = threadIdx.x; e < P * nx; e += blockDim.x) {
        const int rp = L.divn(e), x = e - rp * nx;
        if (rp0 + rp >= npairs) continue;
        const long long row = 2LL * (rp0 + rp);
        T Xr[2], pr[2][3], er[2][3];
        if (mode == XM_PHYS2 || mode == XM_PHYS2R) {
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
                if (Ereal) {
                    const T* b = Ereal + (long long)v * g.N + row * nx + x;
                    er[0][v] = b[0];
                    er[1][v] = b[nx];
                } else if (ph.elastic) {
                    const T2 z = RS[(rp * 3 + v) * ls + skew<true>(x)];
                    er[0][v] = z.x;
                    er[1][v] = z.y;
                } else {
                    er[0][v] = 0;
                    er[1][v] = 0;
                }
            }
        } else {
            const T2 zX = RS[(rp * 4 + 0) * ls + skew<true>(x)];
            Xr[0] = zX.x;
            Xr[1] = zX.y;
#pragma unroll
            for (int v = 0; v < 3; ++v) {
                const T2 z = RS[(rp * 4 + 1 + v) * ls + skew<true>(x)];
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
            for (int r = 0; r < 2; ++r) {
                if (pt.obst)
                    Pt::rhs<T, true>(pt, Xr[r], pr[r], er[r], q[r], gv[r]);
                else
                    Pt::rhs<T, false>(pt, Xr[r], pr[r], er[r], q[r], gv[r]);
            }
            OS[(rp * 4 + 0) * ls + skew<true>(x)] = T2{q[0], q[1]};
#pragma unroll
            for (int v = 0; v < 3; ++v) OS[(rp * 4 + 1 + v) * ls + skew<true>(x)] = T2{gv[0][v], gv[1][v]};
        } else {
            // h(phi_v) lines for the elastic contraction (and the local energy)
#pragma unroll
            for (int v = 0; v < 3; ++v) OS[(rp * 3 + v) * ls + skew<true>(x)] = T2{hfun(pr[0][v]), hfun(pr[1][v])};
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
                    if (ph.obst) {
                        const double S = p[0] + p[1] + p[2];
                        loc = ph.wbar * S * (1.0 - S);
                    } else {
                        for (int v = 0; v < 3; ++v) loc += ph.wbar * p[v] * p[v] * (1.0 - p[v]) * (1.0 - p[v]);
                    }
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
    T2* res = x_fft<-1, PID, R16>(OS, RS, g.px, Fout * P, ls);
    r2c_store<NX>(g, res, ls, Fout, P, rp0, npairs, out);
}

template <typename T>
static int x_rows(const Geo& g) {
    using T2 = typename Cx<T>::t;
    int Pmax = (int)(64 * 1024 / (8 * (size_t)skewed_len(g.nx) * sizeof(T2)));
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

int launch_x_fused(const Geo& g, const Phys& ph, int mode, const void* in, void* out, void* R, const void* Rin,
                   double* partials, double rtol, double atol, cudaStream_t s);

template <typename T>
int launch_x_pass(const Geo& g, const Phys& ph, int mode, const void* in, void* out, void* R, const void* Rin,
                  double* partials, double rtol, double atol, const double* real_in, double* real_out,
                  cudaStream_t s) {
    using T2 = typename Cx<T>::t;
    if constexpr (sizeof(T) == 4) {
        const int nbf = launch_x_fused(g, ph, mode, in, out, R, Rin, partials, rtol, atol, s);
        if (nbf > 0) return nbf;
    }
    const int P = x_rows<T>(g);
    const size_t sm = 2 * 4 * (size_t)P * skewed_len(g.nx) * sizeof(T2);
    const int npairs = g.nz * g.ny / 2;
    const int nb = (npairs + P - 1) / P;
#define PF_XLAUNCH(R16_, PID_)                                                                                       \
    set_smem(k_x_pass<T, R16_, PID_>, sm);                                                                         \
    k_x_pass<T, R16_, PID_><<<nb, kThreads, sm, s>>>(g, ph, mode, reinterpret_cast<const T2*>(in),                 \
                                                     reinterpret_cast<T2*>(out), reinterpret_cast<T*>(R),          \
                                                     reinterpret_cast<const T*>(Rin), partials, rtol, atol, real_in, \
                                                     real_out, P)
    switch (fixed_plan_id(g.px)) {
        case 1: PF_XLAUNCH(false, 1); break;
        case 2: PF_XLAUNCH(false, 2); break;
        case 3: PF_XLAUNCH(false, 3); break;
        case 4: PF_XLAUNCH(false, 4); break;
        case 5: PF_XLAUNCH(false, 5); break;
        case 6: PF_XLAUNCH(false, 6); break;
        case 7: PF_XLAUNCH(false, 7); break;
        case 8: PF_XLAUNCH(false, 8); break;
        case 9: PF_XLAUNCH(false, 9); break;
        case 10: PF_XLAUNCH(false, 10); break;
        case 11: PF_XLAUNCH(false, 11); break;
        default: PF_R16_SWITCH(g.px.has16, PF_XLAUNCH(R16C, 0)); break;
    }
#undef PF_XLAUNCH
    return nb;
}

}  // namespace pf
