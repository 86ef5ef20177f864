// Register-resident x pass of the FFT matvec for padded x lengths of 64 and
// 128 points (FP32).
//
// For every (system, ky, kz) the x pass transforms the three components of
// U along x, multiplies by the symmetric D-hat tensor and transforms back
// (the middle of the zero-padded convolution: IFFT(D-hat . FFT(u))).  Here a
// thread owns the same x positions of all three components of its line, so
// the D-hat product needs no exchange between threads.  The transforms are
// 64-point register FFTs (fft_warp.cuh: lane q + 4p holds elements p + 8r,
// one warp-private transpose per transform).
//
// The lattice fills at most half of every x line (Mx = 64 for Nx = 31, 32;
// Mx = 128 for Nx = 64).  Mx = 64: the four lines q of a warp are four kz
// columns, and the forward transform reads half its registers.  Mx = 128: a
// line of Nx <= 64 inputs x_n has the 128-point spectrum
//   X_{2k} = sum_n x_n w64^{nk},  X_{2k+1} = sum_n (x_n w128^n) w64^{nk},
// and the first 64 outputs of the inverse are
//   y_n = sum_k Y_{2k} w64^{-nk} + w128^{-n} sum_k Y_{2k+1} w64^{-nk},
// so lines q = c + 2h of a warp are two kz columns c and two frequency
// parities h: every lane runs 64-point transforms, and partner lanes (h = 0,
// 1) add their halves of y with one shuffle.
//
// D-hat comes from an FP32 copy laid out for this pass, Dx[slot][ky'][kz'][6][kx']
// on the octant k' <= M/2: the lanes of a line read consecutive kx' of one
// component, so every load moves whole sectors; the off-diagonal components
// change sign under k -> M - k in the axes they name.
#include "fft_warp.cuh"
#include "kernels.h"

namespace eels {

constexpr int XR_WARPS = 4;
constexpr int XR_THREADS = 32 * XR_WARPS;

template <int MX> struct XReg {
    static constexpr bool SPLIT = MX == 128;
    static constexpr int LPW = SPLIT ? 2 : 4;           // kz columns per warp
    static constexpr int KZB = LPW * XR_WARPS;          // kz columns per block
};

template <int MX>
__global__ void __launch_bounds__(XR_THREADS, 4) k_xpass_reg(LatticeDev L, MatvecArgs<float> a) {
    using X = XReg<MX>;
    constexpr bool SPLIT = X::SPLIT;
    __shared__ float2 tws[MX];                          // exp(-2 pi i t / MX)
    __shared__ float2 tiles[XR_WARPS][R64_TILE];
    const int s = blockIdx.z;
    if (a.active && !a.active[s]) return;
    const int ky = blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, q = lane & 3, p = lane >> 2;
    const int h = SPLIT ? (q >> 1) : 0;                 // frequency parity (Mx = 128)
    const int kz = blockIdx.x * X::KZB + warp * X::LPW + (SPLIT ? (q & 1) : q);
    const int Mz = L.Mz, Nx = L.Nx;
    for (int t = threadIdx.x; t < MX; t += XR_THREADS) tws[t] = L.tw32x[t];
    __syncthreads();
    float2* tile = tiles[warp];
    auto tw = [&](int k) { return tws[(MX / 64) * p * k]; };   // w64^(p k)

    const size_t plane = (size_t)Nx * Mz;
    const size_t cstride = (size_t)L.My * plane;
    float2* U0 = a.U + ((size_t)s * 3 * L.My + ky) * plane + kz;
    float2 v[3][8];
    const float2 zero = make_float2(0.f, 0.f);
    constexpr int RIN = SPLIT ? 8 : 4;                  // registers that can hold lattice rows
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int ix = p + 8 * r;
            v[c][r] = (r < RIN && ix < Nx) ? U0[c * cstride + (size_t)ix * Mz] : zero;
        }
    if constexpr (SPLIT) {                              // odd frequencies: x_n w128^n
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const float2 w = h ? tws[p + 8 * r] : make_float2(1.f, 0.f);
#pragma unroll
            for (int c = 0; c < 3; ++c) v[c][r] = v[c][r] * w;
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) fft64_warp_t<false, !SPLIT>(v[c], tile, q, p, tw);

    // D-hat product at kx = p + 8m (Mx = 64) or 2 (p + 8m) + h (Mx = 128); the
    // octant index, and the sign sx of the odd components: -1 for m >= 4,
    // where kx >= MX/2 (at kx = MX/2 those components vanish)
    const int hy = L.My / 2, hz = Mz / 2;
    const int kyr = ky <= hy ? ky : L.My - ky;
    const int kzr = kz <= hz ? kz : Mz - kz;
    const float sy = ky <= hy ? 1.f : -1.f, sz = kz <= hz ? 1.f : -1.f, syz = sy * sz;
    const int Hx = L.Hx;
    const float2* Dk = a.Dx + (((size_t)a.sys_slot[s] * L.Hy + kyr) * L.Hz + kzr) * 6 * Hx;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const int kx = SPLIT ? 2 * (p + 8 * m) + h : p + 8 * m;
        const int kxr = m < 4 ? kx : MX - kx;
        const float sx = m < 4 ? 1.f : -1.f;
        const float2* d = Dk + kxr;
        const float2 dxx = __ldg(d);
        const float2 dxy = (sx * sy) * __ldg(d + Hx);
        const float2 dxz = (sx * sz) * __ldg(d + 2 * Hx);
        const float2 dyy = __ldg(d + 3 * Hx);
        const float2 dyz = syz * __ldg(d + 4 * Hx);
        const float2 dzz = __ldg(d + 5 * Hx);
        const float2 Xv = v[0][m], Yv = v[1][m], Zv = v[2][m];
        v[0][m] = dxx * Xv + dxy * Yv + dxz * Zv;
        v[1][m] = dxy * Xv + dyy * Yv + dyz * Zv;
        v[2][m] = dxz * Xv + dyz * Yv + dzz * Zv;
    }

#pragma unroll
    for (int c = 0; c < 3; ++c) fft64_warp_t<true, false>(v[c], tile, q, p, tw);
    if constexpr (SPLIT) {
        // y_n = z0_n + w128^(-n) z1_n: the h = 1 lane twiddles its z1, lane
        // h = 0 stores rows r < 4 and lane h = 1 rows r >= 4, each receiving
        // the partner's half with one shuffle
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            float2 w = h ? tws[p + 8 * r] : make_float2(1.f, 0.f);
            w.y = -w.y;
#pragma unroll
            for (int c = 0; c < 3; ++c) v[c][r] = v[c][r] * w;
        }
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float2 send = h ? v[c][j] : v[c][j + 4];
                const float2 mine = h ? v[c][j + 4] : v[c][j];
                float2 got;
                got.x = __shfl_xor_sync(0xffffffffu, send.x, 2);
                got.y = __shfl_xor_sync(0xffffffffu, send.y, 2);
                const int ix = p + 8 * (j + 4 * h);
                if (ix < Nx) U0[c * cstride + (size_t)ix * Mz] = mine + got;
            }
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int ix = p + 8 * r;
                if (ix < Nx) U0[c * cstride + (size_t)ix * Mz] = v[c][r];
            }
    }
}

// FP32 copy of the octant D-hat for the register x pass:
// Dx[slot][ky][kz][comp][kx] from Dr64[slot][comp][ky][kx][kz].
__global__ void k_dhat_interleave(LatticeDev L, int n_slot, const double2* __restrict__ Dr64, float2* __restrict__ Dx) {
    const size_t R = (size_t)L.Hx * L.Hy * L.Hz;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= R * 6 * n_slot) return;
    const int kx = (int)(idx % L.Hx);
    const size_t t = idx / L.Hx;                     // ((slot * Hy + ky) * Hz + kz) * 6 + comp
    const int comp = (int)(t % 6);
    const int kz = (int)((t / 6) % L.Hz);
    const size_t sy = t / (6 * (size_t)L.Hz);        // slot * Hy + ky
    const int ky = (int)(sy % L.Hy);
    const size_t slot = sy / L.Hy;
    const double2 v = Dr64[((slot * 6 + comp) * L.Hy + ky) * (size_t)L.Hx * L.Hz + (size_t)kx * L.Hz + kz];
    Dx[idx] = to_f(v);
}

bool xpass_reg_supported(const LatticeDev& L) {
    if (L.Mx == 64) return 2 * L.Nx <= 64 && L.Mz % XReg<64>::KZB == 0;
    if (L.Mx == 128) return 2 * L.Nx <= 128 && L.Mz % XReg<128>::KZB == 0;
    return false;
}

bool launch_xpass_reg(const LatticeDev& L, const MatvecArgs<float>& a, cudaStream_t st) {
    if (!a.Dx || !xpass_reg_supported(L)) return false;
    count_launch();
    if (L.Mx == 64) k_xpass_reg<64><<<dim3(L.Mz / XReg<64>::KZB, L.My, a.S), XR_THREADS, 0, st>>>(L, a);
    else k_xpass_reg<128><<<dim3(L.Mz / XReg<128>::KZB, L.My, a.S), XR_THREADS, 0, st>>>(L, a);
    return true;
}

void launch_dhat_interleave(const LatticeDev& L, int n_slot, const double2* Dr64, float2* Dx, cudaStream_t st) {
    const size_t n = (size_t)L.Hx * L.Hy * L.Hz * 6 * n_slot;
    count_launch();
    k_dhat_interleave<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(L, n_slot, Dr64, Dx);
}

}  // namespace eels
