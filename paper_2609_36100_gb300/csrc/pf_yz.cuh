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
    cols_fft<SIGN, TX, true, 0, R16, PID>(g.py, A, B, src, dst);
}

template <typename T>
void launch_y_pass(const Geo& g, void* buf, int nf, int sign, cudaStream_t s) {
    using T2 = typename Cx<T>::t;
    const int TX = tuned_cols<T>(g, g.tx_y, g.ny, 2, 128 * 1024);
    // a transform of at most two stages never touches its second buffer
    // (stage 0 reads global, the last stage writes global): half the shared
    // memory, more CTAs per SM
    const size_t sm = (g.py.nst <= 2 ? 1 : 2) * (size_t)TX * g.ny * sizeof(T2);
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
    cols_fft<SIGN, TX, true, 0, R16, PID>(g.pz, A, B, src, dst);
}

template <typename T>
void launch_z_pass(const Geo& g, void* buf, int nf, int sign, cudaStream_t s) {
    using T2 = typename Cx<T>::t;
    const int TX = tuned_cols<T>(g, g.tx_zf, g.nz, 2, 128 * 1024);
    const size_t sm = (g.pz.nst <= 2 ? 1 : 2) * (size_t)TX * g.nz * sizeof(T2);  // as in the y pass
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
    cols_fft<-1, TX, false, 0, R16, PID>(g.pz, A, B, src, dst);
}

template <typename T>
void launch_z_fwd(const Geo& g, const Phys& ph, const void* W, void* out, int scale_mode, cudaStream_t s, int nf) {
    using T2 = typename Cx<T>::t;
    const int TX = tuned_cols<T>(g, g.tx_zf, g.nz, 2, 128 * 1024);
    const size_t sm = (g.pz.nst <= 2 ? 1 : 2) * (size_t)TX * g.nz * sizeof(T2);  // as in the y pass
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

template <typename T>
void launch_z_elastic(const Geo& g, const Phys& ph, void* H, cudaStream_t s) {
    using T2 = typename Cx<T>::t;
    const int TX = tuned_cols<T>(g, g.tx_el, g.nz, 4, 128 * 1024);
    const size_t sm = 4 * (size_t)TX * g.nz * sizeof(T2);
    dim3 grid((g.nxh + TX - 1) / TX, g.ny, 1);
    PF_COL_SWITCH8(T, g.pz, TX, set_smem(k_z_elastic<T, TXC, R16C, PIDC>, sm);
                  k_z_elastic<T, TXC, R16C, PIDC><<<grid, kThreads, sm, s>>>(g, ph, reinterpret_cast<T2*>(H)));
}

}  // namespace pf
