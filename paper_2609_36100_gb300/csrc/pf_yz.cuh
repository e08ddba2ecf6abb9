// Strided column passes along y (inverse/forward FFT) and the spectral z
// passes: forward FFT with the k-space scaling of f^E, and the elastic
// Green's contraction between a forward and an inverse FFT along z.
#pragma once
#include "pf_common.cuh"

namespace pf {
// ---------------------------------------------------------------------------
// y pass: in-place complex FFT along y of nf fields
// ---------------------------------------------------------------------------
template <typename T, int SIGN, int TX, bool R16, int PID>
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
    cols_fft<SIGN, TX, true, 0, R16, PID, true>(g.py, A, B, src, dst);
}

template <typename T>
void launch_y_pass(const Geo& g, void* buf, int nf, int sign, cudaStream_t s) {
    using T2 = typename Cx<T>::t;
    const int TX = tuned_cols<T>(g, g.tx_y, g.ny, 2, 128 * 1024);
    // a transform of at most two stages never touches its second buffer
    // (stage 0 reads global, the last stage writes global), and a compiled
    // plan runs its middle stages in place: half the shared memory, more
    // CTAs per SM
    const size_t sm = col_buffers<T>(g.py, TX) * (size_t)TX * g.ny * sizeof(T2);
    dim3 grid((g.nxh + TX - 1) / TX, g.nz, nf);
    if (sign > 0) {
        PF_COL_SWITCH(T, g.py, TX, set_smem(k_y_pass<T, 1, TXC, R16C, PIDC>, sm);
                      k_y_pass<T, 1, TXC, R16C, PIDC><<<grid, kThreads, sm, s>>>(g, reinterpret_cast<T2*>(buf)));
    } else {
        PF_COL_SWITCH(T, g.py, TX, set_smem(k_y_pass<T, -1, TXC, R16C, PIDC>, sm);
                      k_y_pass<T, -1, TXC, R16C, PIDC><<<grid, kThreads, sm, s>>>(g, reinterpret_cast<T2*>(buf)));
    }
}

// ---------------------------------------------------------------------------
// z pass: in-place FFT along z of nf fields (the inverse transform of an
// assembled FP32-bulk stage)
// ---------------------------------------------------------------------------
template <typename T, int SIGN, int TX, bool R16, int PID>
__global__ void __launch_bounds__(kThreads) k_z_pass(Geo g, typename Cx<T>::t* __restrict__ buf) {
    PF_SKIP_INACTIVE(g);
    using T2 = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smraw[];
    T2* A = reinterpret_cast<T2*>(smraw);
    T2* B = A + TX * g.nz;
    const int f = blockIdx.z, ky = blockIdx.y, kx0 = blockIdx.x * TX;
    const int ncol = min(TX, g.nxh - kx0);
    T2* base = buf + (long long)f * g.NK + (long long)ky * g.nxh + kx0;
    const long long zs = (long long)g.ny * g.nxh;
    auto src = [&](int kz, int col) -> T2 { return col < ncol ? base[kz * zs + col] : T2{0, 0}; };
    auto dst = [&](int kz, int col, T2 v) {
        if (col < ncol) base[kz * zs + col] = v;
    };
    cols_fft<SIGN, TX, true, 0, R16, PID, true>(g.pz, A, B, src, dst);
}

template <typename T>
void launch_z_pass(const Geo& g, void* buf, int nf, int sign, cudaStream_t s) {
    using T2 = typename Cx<T>::t;
    const int TX = tuned_cols<T>(g, g.tx_zf, g.nz, 2, 128 * 1024);
    const size_t sm = col_buffers<T>(g.pz, TX) * (size_t)TX * g.nz * sizeof(T2);  // as in the y pass
    dim3 grid((g.nxh + TX - 1) / TX, g.ny, nf);
    if (sign > 0) {
        PF_COL_SWITCH(T, g.pz, TX, set_smem(k_z_pass<T, 1, TXC, R16C, PIDC>, sm);
                      k_z_pass<T, 1, TXC, R16C, PIDC><<<grid, kThreads, sm, s>>>(g, reinterpret_cast<T2*>(buf)));
    } else {
        PF_COL_SWITCH(T, g.pz, TX, set_smem(k_z_pass<T, -1, TXC, R16C, PIDC>, sm);
                      k_z_pass<T, -1, TXC, R16C, PIDC><<<grid, kThreads, sm, s>>>(g, reinterpret_cast<T2*>(buf)));
    }
}

// ---------------------------------------------------------------------------
// z pass, forward: FFT along z then k-space scaling (the last stage's store)
//   mode 0: y^ = W / N  -> FP64                                  (set_state)
//   mode 1: f^E_X = -M k^2 q^/N, f^E_phi = -L g^/N -> compute type (stages)
//   mode 2: same scaling -> FP64                                  (ABI f^E)
// ---------------------------------------------------------------------------
template <typename T, typename OT2, int TX, bool R16, int PID>
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
    const double invN = g.invN;
    const T mN = phys_t<T>(ph).mN, lN = phys_t<T>(ph).lN;
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
    cols_fft<-1, TX, false, 0, R16, PID, true>(g.pz, A, B, src, dst);
}

template <typename T>
void launch_z_fwd(const Geo& g, const Phys& ph, const void* W, void* out, int scale_mode, cudaStream_t s, int nf) {
    using T2 = typename Cx<T>::t;
    const int TX = tuned_cols<T>(g, g.tx_zf, g.nz, 2, 128 * 1024);
    // modes 0/2 run the generic stages (two buffers for three or more stages)
    const size_t sm = (scale_mode == 1 ? col_buffers<T>(g.pz, TX) : (g.pz.nst <= 2 ? 1 : 2)) * (size_t)TX * g.nz *
                      sizeof(T2);
    dim3 grid((g.nxh + TX - 1) / TX, g.ny, nf);
    if (scale_mode == 1) {
        PF_COL_SWITCH(T, g.pz, TX, set_smem(k_z_fwd<T, T2, TXC, R16C, PIDC>, sm);
                      k_z_fwd<T, T2, TXC, R16C, PIDC><<<grid, kThreads, sm, s>>>(
                          g, ph, reinterpret_cast<const T2*>(W), reinterpret_cast<T2*>(out), 1));
    } else {
        constexpr int PIDC = 0;  // FP64 output (state in, ABI f^E): generic stages
        PF_R16_SWITCH(g.pz.has16, PF_TX_SWITCH(TX, set_smem(k_z_fwd<T, double2, TXC, R16C, PIDC>, sm);
                     k_z_fwd<T, double2, TXC, R16C, PIDC><<<grid, kThreads, sm, s>>>(
                         g, ph, reinterpret_cast<const T2*>(W), reinterpret_cast<double2*>(out), scale_mode)))
    }
}

template <typename T, int TX, bool R16, int PID>
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
    bool nst_even;
    if constexpr (PID > 0)
        nst_even = RadInfo<typename FixedPlan<PID>::Rad>::count % 2 == 0;
    else
        nst_even = (g.pz.nst % 2) == 0;
    // forward transforms: global -> field slot (middle stages ping-pong with E
    // so that the last stage reads E and writes the slot)
#pragma unroll 1
    for (int f = 0; f < 3; ++f) {
        T2* S = slot[f];
        const long long fb = (long long)f * g.NK + rowoff;
        auto src = [&](int kz, int col) -> T2 { return col < ncol ? H[fb + kz * zs + col] : T2{0, 0}; };
        auto dst = [&](int kz, int col, T2 v) { S[kz * TX + col] = v; };
        if (nst_even)
            cols_fft<-1, TX, false, 0, R16, PID>(g.pz, E, S, src, dst);
        else
            cols_fft<-1, TX, false, 0, R16, PID>(g.pz, S, E, src, dst);
        __syncthreads();
    }
    const T invN = std::is_same<T, float>::value ? (T)g.invN32 : (T)g.invN;
    const PhysT<T>& pt = phys_t<T>(ph);
    const T kyv = kval<T>(g, 1, ky);
    // FP32 contexts with diagonal eigenstrains read B/N from the octant table
    const float* bt = sizeof(T) == 4 ? g.btab : nullptr;
    const int hy = g.ny / 2 + 1;
    const long long tn = (long long)(g.nz / 2 + 1) * hy * g.nxh;
    const long long trow = (long long)(ky <= g.ny / 2 ? ky : g.ny - ky) * g.nxh + kx0;
    for (int r = threadIdx.x; r < tile; r += blockDim.x) {
        const int col = r & (TX - 1), kz = r / TX;
        if (col >= ncol) continue;
        T Bm[3][3];
        T sc = invN;
        if (bt) {
            const long long ti = (long long)(kz <= g.nz / 2 ? kz : g.nz - kz) * hy * g.nxh + trow + col;
            Bm[0][0] = (T)__ldg(bt + ti);
            Bm[0][1] = Bm[1][0] = (T)__ldg(bt + tn + ti);
            Bm[0][2] = Bm[2][0] = (T)__ldg(bt + 2 * tn + ti);
            Bm[1][1] = (T)__ldg(bt + 3 * tn + ti);
            Bm[1][2] = Bm[2][1] = (T)__ldg(bt + 4 * tn + ti);
            Bm[2][2] = (T)__ldg(bt + 5 * tn + ti);
            sc = (T)1;
        } else {
            elastic_kernel<T>(pt, kval<T>(g, 0, kx0 + col), kyv, kval<T>(g, 2, kz), Bm);
        }
        const T2 h0 = slot[0][r], h1 = slot[1][r], h2 = slot[2][r];
        slot[0][r] = T2{(Bm[0][0] * h0.x + Bm[0][1] * h1.x + Bm[0][2] * h2.x) * sc,
                        (Bm[0][0] * h0.y + Bm[0][1] * h1.y + Bm[0][2] * h2.y) * sc};
        slot[1][r] = T2{(Bm[1][0] * h0.x + Bm[1][1] * h1.x + Bm[1][2] * h2.x) * sc,
                        (Bm[1][0] * h0.y + Bm[1][1] * h1.y + Bm[1][2] * h2.y) * sc};
        slot[2][r] = T2{(Bm[2][0] * h0.x + Bm[2][1] * h1.x + Bm[2][2] * h2.x) * sc,
                        (Bm[2][0] * h0.y + Bm[2][1] * h1.y + Bm[2][2] * h2.y) * sc};
    }
    __syncthreads();
    // inverse transforms: field slot -> global (stage 0 reads the slot and
    // writes E)
#pragma unroll 1
    for (int f = 0; f < 3; ++f) {
        T2* S = slot[f];
        const long long fb = (long long)f * g.NK + rowoff;
        auto src = [&](int kz, int col) -> T2 { return S[kz * TX + col]; };
        auto dst = [&](int kz, int col, T2 v) {
            if (col < ncol) H[fb + kz * zs + col] = v;
        };
        cols_fft<+1, TX, false, 0, R16, PID>(g.pz, E, S, src, dst);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Elastic pass with a compile-time plan, one shared tile per CTA: the three
// h fields of TX kx columns stay in one [field][kz][col] tile, transformed in
// place.  The last forward stage (radix R), the Green's contraction and the
// first inverse stage (radix R again: the inverse runs the forward radix
// order reversed, so both stages see the element positions j + (N/R) t) run
// in the registers of one thread per (column, j), which holds all three
// fields of its R wave numbers: no shared-memory round trip and no barrier
// between the forward transform, the contraction and the inverse.  Middle
// stages of longer plans run in place through registers (every load of a
// stage, a barrier, then the stores).  NT = TX N / R threads, one per
// (column, j) of the fused stage.
// ---------------------------------------------------------------------------
// stage from global (first forward stage) or to global (last inverse stage):
// no staging, the tile is written only by loads from global or read only
template <int R, int SIGN, int TX, int N, int NS, int NF, int NT, typename T2, class Ld, class St>
__device__ __forceinline__ void tile_stage_io(const T2* __restrict__ tw, Ld ld, St st) {
    constexpr int M = N / R, JOBS = NF * TX * M, TWS = N / (NS * R);
    for (int idx = threadIdx.x; idx < JOBS; idx += NT) {
        const int f = idx / (TX * M), r = idx - f * (TX * M), col = r % TX, j = r / TX;
        T2 v[R];
#pragma unroll
        for (int t = 0; t < R; ++t) v[t] = ld(f, j + t * M, col);
        const int jq = j / NS, k = j - jq * NS;
        if constexpr (NS > 1) apply_twiddles<R, SIGN>(v, tw, k * TWS);
        Bfly<R, SIGN, T2>::run(v);
        const int base = jq * NS * R + k;
#pragma unroll
        for (int t = 0; t < R; ++t) st(f, base + t * NS, col, v[t]);
    }
}

// in-place stages of a radix list between the first and the last, NS growing
template <int SIGN, int TX, int N, int NS, int NF, int NT, typename T2>
__device__ __forceinline__ void tile_stages_inplace(T2*, const T2*, Radices<>) {}
template <int SIGN, int TX, int N, int NS, int NF, int NT, typename T2, int R, int... Rest>
__device__ __forceinline__ void tile_stages_inplace(T2* S, const T2* tw, Radices<R, Rest...>) {
    tile_stage_inplace<R, SIGN, TX, N, NS, NF, NT>(S, tw);
    tile_stages_inplace<SIGN, TX, N, NS * R, NF, NT>(S, tw, Radices<Rest...>{});
}

// CTAs per SM the register budget is planned for: 128 registers a thread
// where the fused stage holds few values, the full file for one CTA where it
// holds 3 x 16 complex values (FP32) or any FP64 tile
template <typename T, int PID, int NT>
constexpr int elastic_min_blocks() {
    constexpr int RL = RadInfo<typename FixedPlan<PID>::Rad>::last;
    constexpr int regs = (RL >= 16 || sizeof(T) == 8) ? 255 : 128;
    return NT * regs <= 65536 ? 65536 / (NT * regs) : 1;
}

template <typename T, int TX, int PID, int NT>
__global__ void __launch_bounds__(NT, elastic_min_blocks<T, PID, NT>())
    k_z_elastic_fused(Geo g, Phys ph, typename Cx<T>::t* __restrict__ H) {
    PF_SKIP_INACTIVE(g);
    using T2 = typename Cx<T>::t;
    using Fwd = typename FixedPlan<PID>::Rad;
    using Inv = Reversed<Fwd>;
    constexpr int N = FixedPlan<PID>::N;
    constexpr int RF = RadInfo<Fwd>::first, RL = RadInfo<Fwd>::last;
    constexpr int M = N / RL;  // the fused stage's butterflies per column
    static_assert(NT == TX * M, "one thread per (column, j) of the fused stage");
    extern __shared__ __align__(16) unsigned char smraw[];
    T2* S = reinterpret_cast<T2*>(smraw);  // [3][N][TX]
    const int ky = blockIdx.y, kx0 = blockIdx.x * TX;
    const int ncol = min(TX, g.nxh - kx0);
    const long long rowoff = (long long)ky * g.nxh + kx0;
    const long long zs = (long long)g.ny * g.nxh;
    const T2* tw = twiddles<T2>(g.pz);
    // forward stage 1: global -> tile
    {
        auto ld = [&](int f, int kz, int col) -> T2 {
            return col < ncol ? H[(long long)f * g.NK + rowoff + kz * zs + col] : T2{0, 0};
        };
        auto st = [&](int f, int kz, int col, T2 v) { S[f * (N * TX) + kz * TX + col] = v; };
        tile_stage_io<RF, -1, TX, N, 1, 3, NT>(tw, ld, st);
    }
    __syncthreads();
    // forward middle stages (in place)
    tile_stages_inplace<-1, TX, N, RF, 3, NT>(S, tw, typename PlanInner<Fwd>::type{});
    // fused: last forward stage, contraction, first inverse stage
    {
        const int col = threadIdx.x % TX, j = threadIdx.x / TX;
        T2 h[3][RL];
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            const T2* src = S + f * (N * TX) + j * TX + col;
#pragma unroll
            for (int t = 0; t < RL; ++t) h[f][t] = src[t * M * TX];
            apply_twiddles<RL, -1>(h[f], tw, j);  // NS = N / RL: k = j, table stride 1
            Bfly<RL, -1, T2>::run(h[f]);
        }
        __syncthreads();
        const T invN = std::is_same<T, float>::value ? (T)g.invN32 : (T)g.invN;
        const PhysT<T>& pt = phys_t<T>(ph);
        const T kxv = kval<T>(g, 0, kx0 + (col < ncol ? col : 0)), kyv = kval<T>(g, 1, ky);
        // FP32 contexts with diagonal eigenstrains read B/N from the table
        // (held in L2 across the tiles); otherwise B is formed per wave vector
        const float* bt = sizeof(T) == 4 ? g.btab : nullptr;
        const int hy = g.ny / 2 + 1, hz = g.nz / 2 + 1;
        const long long tn = (long long)hz * hy * g.nxh;
        const long long trow = (long long)(ky <= g.ny / 2 ? ky : g.ny - ky) * g.nxh + kx0 + (col < ncol ? col : 0);
#pragma unroll
        for (int t = 0; t < RL; ++t) {
            T Bm[3][3];
            T sc = invN;
            if (bt) {
                const int kz = j + t * M;
                const long long ti = (long long)(kz <= g.nz / 2 ? kz : g.nz - kz) * hy * g.nxh + trow;
                Bm[0][0] = (T)__ldg(bt + ti);
                Bm[0][1] = Bm[1][0] = (T)__ldg(bt + tn + ti);
                Bm[0][2] = Bm[2][0] = (T)__ldg(bt + 2 * tn + ti);
                Bm[1][1] = (T)__ldg(bt + 3 * tn + ti);
                Bm[1][2] = Bm[2][1] = (T)__ldg(bt + 4 * tn + ti);
                Bm[2][2] = (T)__ldg(bt + 5 * tn + ti);
                sc = (T)1;
            } else {
                elastic_kernel<T>(pt, kxv, kyv, kval<T>(g, 2, j + t * M), Bm);
            }
            const T2 a = h[0][t], b = h[1][t], c = h[2][t];
#pragma unroll
            for (int v = 0; v < 3; ++v)
                h[v][t] = T2{(Bm[v][0] * a.x + Bm[v][1] * b.x + Bm[v][2] * c.x) * sc,
                             (Bm[v][0] * a.y + Bm[v][1] * b.y + Bm[v][2] * c.y) * sc};
        }
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            Bfly<RL, +1, T2>::run(h[f]);  // first inverse stage: NS = 1, no twiddles
            T2* dst = S + f * (N * TX) + (j * RL) * TX + col;
#pragma unroll
            for (int t = 0; t < RL; ++t) dst[t * TX] = h[f][t];
        }
    }
    __syncthreads();
    // inverse middle stages (in place), then the last inverse stage: tile -> global
    tile_stages_inplace<+1, TX, N, RL, 3, NT>(S, tw, typename PlanInner<Inv>::type{});
    {
        auto ld = [&](int f, int kz, int col) -> T2 { return S[f * (N * TX) + kz * TX + col]; };
        auto st = [&](int f, int kz, int col, T2 v) {
            if (col < ncol) H[(long long)f * g.NK + rowoff + kz * zs + col] = v;
        };
        tile_stage_io<RF, +1, TX, N, N / RF, 3, NT>(tw, ld, st);
    }
}

// Elastic pass with a compile-time plan and no fused stage: the three h
// fields of TX columns share one in-place tile, and every transform stage
// runs over the three fields at once (one job per butterfly of any field,
// NT threads: one per butterfly of the plan's largest radix), so a stage is
// one load phase, one barrier and one store phase for all fields.  Forward
// transform (the first stage reads global memory), the contraction
// e^_v = sum_q (B_vq / N) h^_q in place, the inverse transform (the last
// stage writes global memory).  Fewer registers per thread than the fused
// stage, which holds three fields' values of its butterfly at once.
template <typename T, int TX, int PID, int NT>
__global__ void __launch_bounds__(NT) k_z_elastic_stages(Geo g, Phys ph, typename Cx<T>::t* __restrict__ H) {
    PF_SKIP_INACTIVE(g);
    using T2 = typename Cx<T>::t;
    using Fwd = typename FixedPlan<PID>::Rad;
    using Inv = Reversed<Fwd>;
    constexpr int N = FixedPlan<PID>::N;
    constexpr int RF = RadInfo<Fwd>::first, RL = RadInfo<Fwd>::last;
    extern __shared__ __align__(16) unsigned char smraw[];
    T2* S = reinterpret_cast<T2*>(smraw);  // [3][N][TX]
    const int ky = blockIdx.y, kx0 = blockIdx.x * TX;
    const int ncol = min(TX, g.nxh - kx0);
    const long long rowoff = (long long)ky * g.nxh + kx0;
    const long long zs = (long long)g.ny * g.nxh;
    const T2* tw = twiddles<T2>(g.pz);
    {
        auto ld = [&](int f, int kz, int col) -> T2 {
            return col < ncol ? H[(long long)f * g.NK + rowoff + kz * zs + col] : T2{0, 0};
        };
        auto st = [&](int f, int kz, int col, T2 v) { S[f * (N * TX) + kz * TX + col] = v; };
        tile_stage_io<RF, -1, TX, N, 1, 3, NT>(tw, ld, st);
    }
    __syncthreads();
    // the remaining forward stages, the last one included, in place
    tile_stages_inplace<-1, TX, N, RF, 3, NT>(S, tw, typename DropFirst<Fwd>::type{});
    {
        const T invN = std::is_same<T, float>::value ? (T)g.invN32 : (T)g.invN;
        const PhysT<T>& pt = phys_t<T>(ph);
        const T kyv = kval<T>(g, 1, ky);
        const float* bt = sizeof(T) == 4 ? g.btab : nullptr;
        const int hy = g.ny / 2 + 1;
        const long long tn = (long long)(g.nz / 2 + 1) * hy * g.nxh;
        const long long trow = (long long)(ky <= g.ny / 2 ? ky : g.ny - ky) * g.nxh + kx0;
        for (int e = threadIdx.x; e < N * TX; e += NT) {
            const int kz = e / TX, col = e - kz * TX;
            if (col >= ncol) continue;
            T Bm[3][3];
            T sc = invN;
            if (bt) {
                const long long ti = (long long)(kz <= g.nz / 2 ? kz : g.nz - kz) * hy * g.nxh + trow + col;
                Bm[0][0] = (T)__ldg(bt + ti);
                Bm[0][1] = Bm[1][0] = (T)__ldg(bt + tn + ti);
                Bm[0][2] = Bm[2][0] = (T)__ldg(bt + 2 * tn + ti);
                Bm[1][1] = (T)__ldg(bt + 3 * tn + ti);
                Bm[1][2] = Bm[2][1] = (T)__ldg(bt + 4 * tn + ti);
                Bm[2][2] = (T)__ldg(bt + 5 * tn + ti);
                sc = (T)1;
            } else {
                elastic_kernel<T>(pt, kval<T>(g, 0, kx0 + col), kyv, kval<T>(g, 2, kz), Bm);
            }
            const T2 a = S[e], b = S[N * TX + e], c = S[2 * N * TX + e];
#pragma unroll
            for (int v = 0; v < 3; ++v)
                S[v * N * TX + e] = T2{(Bm[v][0] * a.x + Bm[v][1] * b.x + Bm[v][2] * c.x) * sc,
                                       (Bm[v][0] * a.y + Bm[v][1] * b.y + Bm[v][2] * c.y) * sc};
        }
    }
    __syncthreads();
    // inverse: the reversed radix order (its first stage has NS = 1), in place
    // up to the last stage, which writes global memory
    tile_stage_inplace<RL, +1, TX, N, 1, 3, NT>(S, tw);
    tile_stages_inplace<+1, TX, N, RL, 3, NT>(S, tw, typename PlanInner<Inv>::type{});
    {
        auto ld = [&](int f, int kz, int col) -> T2 { return S[f * (N * TX) + kz * TX + col]; };
        auto st = [&](int f, int kz, int col, T2 v) {
            if (col < ncol) H[(long long)f * g.NK + rowoff + kz * zs + col] = v;
        };
        tile_stage_io<RF, +1, TX, N, N / RF, 3, NT>(tw, ld, st);
    }
}

template <int PID, int TX>
constexpr int elastic_stage_threads() {
    constexpr int n = 3 * TX * FixedPlan<PID>::N / RadMax<typename FixedPlan<PID>::Rad>::value;
    return n > 1024 ? 1024 : (n + 31) / 32 * 32;
}

// compiled plans of two or more stages run the fused elastic pass
template <int PID>
constexpr bool fused_elastic_ok() {
    return PID > 0 && RadInfo<typename FixedPlan<PID>::Rad>::count >= 2;
}

template <typename T, int PID>
static bool launch_z_elastic_fused(const Geo& g, const Phys& ph, void* H, int tuned, cudaStream_t s) {
    using T2 = typename Cx<T>::t;
    if constexpr (!fused_elastic_ok<PID>()) {
        return false;
    } else {
        constexpr int N = FixedPlan<PID>::N;
        constexpr int M = N / RadInfo<typename FixedPlan<PID>::Rad>::last;
        // widest tile (16, 8, 4, 2 columns) with NT <= 1024 threads and at most
        // ~100 KB of shared memory, or the tuned width if it fits
        auto fits = [&](int tx) { return tx * M <= 1024 && 3 * (size_t)tx * N * sizeof(T2) <= 100 * 1024; };
        int TX = 0;
        for (int tx : {16, 8, 4, 2})
            if (fits(tx) && (TX == 0 || (tuned > 0 && tx == tuned))) TX = tx;
        if (tuned <= 0)
            for (int tx : {16, 8, 4, 2})
                if (fits(tx) && tx / 2 < g.nxh) {
                    TX = tx;
                    break;
                }
        if (TX == 0) return false;
        const size_t sm = 3 * (size_t)TX * N * sizeof(T2);
        dim3 grid((g.nxh + TX - 1) / TX, g.ny, 1);
#define PF_ELF(TXC)                                                                                       if constexpr ((TXC) * M <= 1024) {                                                                        set_smem(k_z_elastic_fused<T, TXC, PID, (TXC) * M>, sm);                                              k_z_elastic_fused<T, TXC, PID, (TXC) * M><<<grid, (TXC) * M, sm, s>>>(g, ph, reinterpret_cast<T2*>(H));     }
        switch (TX) {
            case 16: PF_ELF(16); break;
            case 8: PF_ELF(8); break;
            case 4: PF_ELF(4); break;
            default: PF_ELF(2); break;
        }
#undef PF_ELF
        return true;
    }
}

#ifdef PF_ELASTIC_ALT_TU
// the compiled-plan elastic pass with every stage over the three fields (no
// fused stage): tile width as for the fused form
template <typename T, int PID>
static bool launch_z_elastic_unf(const Geo& g, const Phys& ph, void* H, int tuned, cudaStream_t s) {
    using T2 = typename Cx<T>::t;
    if constexpr (!fused_elastic_ok<PID>()) {
        return false;
    } else {
        constexpr int N = FixedPlan<PID>::N;
        auto fits = [&](int tx) { return 3 * (size_t)tx * N * sizeof(T2) <= 100 * 1024; };
        int TX = 0;
        for (int tx : {16, 8, 4, 2})
            if (fits(tx) && (TX == 0 || (tuned > 0 && tx == tuned))) TX = tx;
        if (tuned <= 0)
            for (int tx : {16, 8, 4, 2})
                if (fits(tx) && tx / 2 < g.nxh) {
                    TX = tx;
                    break;
                }
        if (TX == 0) return false;
        const size_t sm = 3 * (size_t)TX * N * sizeof(T2);
        dim3 grid((g.nxh + TX - 1) / TX, g.ny, 1);
#define PF_ELU(TXC)                                                                                   \
    {                                                                                                 \
        constexpr int NTU = elastic_stage_threads<PID, TXC>();                                        \
        set_smem(k_z_elastic_stages<T, TXC, PID, NTU>, sm);                                           \
        k_z_elastic_stages<T, TXC, PID, NTU><<<grid, NTU, sm, s>>>(g, ph, reinterpret_cast<T2*>(H));  \
    }
        switch (TX) {
            case 16: PF_ELU(16); break;
            case 8: PF_ELU(8); break;
            case 4: PF_ELU(4); break;
            default: PF_ELU(2); break;
        }
#undef PF_ELU
        return true;
    }
}

template <typename T>
bool launch_z_elastic_unfused(const Geo& g, const Phys& ph, void* H, int pid, cudaStream_t s) {
    switch (pid) {
        case 1: return launch_z_elastic_unf<T, 1>(g, ph, H, g.tx_el, s);
        case 2: return launch_z_elastic_unf<T, 2>(g, ph, H, g.tx_el, s);
        case 3: return launch_z_elastic_unf<T, 3>(g, ph, H, g.tx_el, s);
        case 4: return launch_z_elastic_unf<T, 4>(g, ph, H, g.tx_el, s);
        case 5: return launch_z_elastic_unf<T, 5>(g, ph, H, g.tx_el, s);
        case 6: return launch_z_elastic_unf<T, 6>(g, ph, H, g.tx_el, s);
        case 7: return launch_z_elastic_unf<T, 7>(g, ph, H, g.tx_el, s);
        case 8: return launch_z_elastic_unf<T, 8>(g, ph, H, g.tx_el, s);
        case 9: return launch_z_elastic_unf<T, 9>(g, ph, H, g.tx_el, s);
        case 10: return launch_z_elastic_unf<T, 10>(g, ph, H, g.tx_el, s);
        case 11: return launch_z_elastic_unf<T, 11>(g, ph, H, g.tx_el, s);
        default: return false;
    }
}
#endif

template <typename T>
void launch_z_elastic(const Geo& g, const Phys& ph, void* H, cudaStream_t s) {
    using T2 = typename Cx<T>::t;
    bool done = false;
    // el_pid < 0: the one-kernel pass with the column transforms of the z
    // axis (no fused stage), also where a compiled plan exists
    if (g.el_pid >= 0 && g.pz.n == g.nz && g.nz >= 32) {
        const int pid = (g.el_pid > 0 && fixed_plan_len(g.el_pid) == g.nz) ? g.el_pid : fixed_plan_id(g.pz);
        if (g.el_unfused == 2 && launch_z_elastic_cluster<T>(g, ph, H, pid, s)) return;
        if (g.el_unfused == 1 && launch_z_elastic_unfused<T>(g, ph, H, pid, s)) return;
        switch (pid) {
            case 1: done = launch_z_elastic_fused<T, 1>(g, ph, H, g.tx_el, s); break;
            case 2: done = launch_z_elastic_fused<T, 2>(g, ph, H, g.tx_el, s); break;
            case 3: done = launch_z_elastic_fused<T, 3>(g, ph, H, g.tx_el, s); break;
            case 4: done = launch_z_elastic_fused<T, 4>(g, ph, H, g.tx_el, s); break;
            case 5: done = launch_z_elastic_fused<T, 5>(g, ph, H, g.tx_el, s); break;
            case 6: done = launch_z_elastic_fused<T, 6>(g, ph, H, g.tx_el, s); break;
            case 7: done = launch_z_elastic_fused<T, 7>(g, ph, H, g.tx_el, s); break;
            case 8: done = launch_z_elastic_fused<T, 8>(g, ph, H, g.tx_el, s); break;
            case 9: done = launch_z_elastic_fused<T, 9>(g, ph, H, g.tx_el, s); break;
            case 10: done = launch_z_elastic_fused<T, 10>(g, ph, H, g.tx_el, s); break;
            case 11: done = launch_z_elastic_fused<T, 11>(g, ph, H, g.tx_el, s); break;
            default: break;
        }
    }
    if (done) return;
    const int TX = tuned_cols<T>(g, g.tx_el, g.nz, 4, 128 * 1024);
    const size_t sm = 4 * (size_t)TX * g.nz * sizeof(T2);
    dim3 grid((g.nxh + TX - 1) / TX, g.ny, 1);
    PF_COL_SWITCH8(T, g.pz, TX, set_smem(k_z_elastic<T, TXC, R16C, PIDC>, sm);
                  k_z_elastic<T, TXC, R16C, PIDC><<<grid, kThreads, sm, s>>>(g, ph, reinterpret_cast<T2*>(H)));
}

}  // namespace pf
