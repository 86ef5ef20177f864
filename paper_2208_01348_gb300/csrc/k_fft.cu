// FFT kernels of the DDA matrix-vector product and of the D-hat build.
//
// The interaction sum conv(u)_i = sum_{j != i} G~'(r_i - r_j) u_j over a
// cubic lattice is a 3-D convolution; embedding it in a circulant of
// extents M >= 2N - 1 per axis turns it into  IFFT( D-hat . FFT(u) ), where
// D-hat is the FFT of the six symmetric components of G~' on the padded
// lattice (separation (i - M) for the upper indices, zero at R = 0 and at
// indices no separation reaches).  The input u is non-zero only on the
// first Nx x Ny x Nz corner and only that corner of the output is needed, so
// the forward transform runs z (Nx*Ny lines), then y (Nx*Mz lines), then x
// (My*Mz lines, fused with the D-hat product and the inverse x transform),
// and the inverse retraces y then z:  five passes over one scratch array
// U[s][c][y][x][z] (z fastest), every pass coalesced along z or x.
//
// D-hat is stored on the octant 0 <= k <= M/2 only (6 (M/2+1)^3 values):
// the diagonal components are even in each k and xy, xz, yz are odd in the
// two axes they name, so D(M - k) = +-D(k).
#include <algorithm>
#include <cstdio>

#include "fft_warp.cuh"
#include "kernels.h"

namespace eels {

constexpr int FFT_THREADS = 256;

template <typename Rl> __device__ __forceinline__ const cx<Rl>* tw_of(const LatticeDev& L, int axis);
template <> __device__ __forceinline__ const double2* tw_of<double>(const LatticeDev& L, int axis) {
    return axis == 0 ? L.tw64x : (axis == 1 ? L.tw64y : L.tw64z);
}
template <> __device__ __forceinline__ const float2* tw_of<float>(const LatticeDev& L, int axis) {
    return axis == 0 ? L.tw32x : (axis == 1 ? L.tw32y : L.tw32z);
}

// ---------------------------------------------------------------------------
// Pass 1 (five-pass path): scatter the dipole vector onto the lattice (times
// coef) and transform along z.  Block: W y-adjacent lines at fixed (s, c, ix).
// ---------------------------------------------------------------------------
template <typename Rl, int W>
__global__ void __launch_bounds__(FFT_THREADS) k_zfwd(LatticeDev L, MatvecArgs<Rl> a) {
    using C = cx<Rl>;
    const int b = blockIdx.z, s = b / 3, c = b % 3;
    if (a.active && !a.active[s]) return;
    const int ix = blockIdx.y, iy0 = blockIdx.x * W;
    const int Mz = L.Mz, ls = Mz + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* A = tw + Mz;
    C* B = A + W * ls;
    const C* twg = tw_of<Rl>(L, 2);
    for (int t = threadIdx.x; t < Mz; t += blockDim.x) tw[t] = twg[t];
    const C* xs = a.x + ((size_t)s * 3 + c) * L.N;
    const double2* cf = a.coef + (size_t)s * EELS_MAX_MAT;
    for (int t = threadIdx.x; t < W * Mz; t += blockDim.x) {
        const int iz = t % Mz, w = t / Mz, iy = iy0 + w;
        C v = mk<C>(0.0, 0.0);
        if (iz < L.Nz && iy < L.Ny) {
            const int dip = L.cellmap[((size_t)ix * L.Ny + iy) * L.Nz + iz];
            if (dip >= 0) v = xs[dip] * cvt<C>(cf[L.mat[dip]]);
        }
        A[w * ls + iz] = v;
    }
    __syncthreads();
    const C* r = fft_lines<false, false, W>(A, B, ls, 1, L.pz, tw);
    C* U = a.U + (((size_t)s * 3 + c) * L.My * L.Nx + ix) * (size_t)Mz;
    const size_t row = (size_t)L.Nx * Mz;
    for (int t = threadIdx.x; t < W * Mz; t += blockDim.x) {
        const int kz = t % Mz, w = t / Mz, iy = iy0 + w;
        if (iy < L.Ny) U[(size_t)iy * row + kz] = r[w * ls + kz];
    }
}

// ---------------------------------------------------------------------------
// Pass 5 (five-pass path): inverse z transform and gather:
//   y = diag x - coef conv / M.
// ---------------------------------------------------------------------------
template <typename Rl, int W>
__global__ void __launch_bounds__(FFT_THREADS) k_zinv(LatticeDev L, MatvecArgs<Rl> a, Rl invM) {
    using C = cx<Rl>;
    const int b = blockIdx.z, s = b / 3, c = b % 3;
    if (a.active && !a.active[s]) return;
    const int ix = blockIdx.y, iy0 = blockIdx.x * W;
    const int Mz = L.Mz, ls = Mz + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* A = tw + Mz;
    C* B = A + W * ls;
    const C* twg = tw_of<Rl>(L, 2);
    for (int t = threadIdx.x; t < Mz; t += blockDim.x) tw[t] = twg[t];
    const C* U = a.U + (((size_t)s * 3 + c) * L.My * L.Nx + ix) * (size_t)Mz;
    const size_t row = (size_t)L.Nx * Mz;
    for (int t = threadIdx.x; t < W * Mz; t += blockDim.x) {
        const int kz = t % Mz, w = t / Mz, iy = iy0 + w;
        A[w * ls + kz] = iy < L.Ny ? U[(size_t)iy * row + kz] : mk<C>(0.0, 0.0);
    }
    __syncthreads();
    const C* r = fft_lines<true, false, W>(A, B, ls, 1, L.pz, tw);
    const C* xs = a.x + ((size_t)s * 3 + c) * L.N;
    C* ys = a.y + ((size_t)s * 3 + c) * L.N;
    const double2* cf = a.coef + (size_t)s * EELS_MAX_MAT;
    const double2* dg = a.diag + (size_t)s * EELS_MAX_MAT;
    for (int t = threadIdx.x; t < W * L.Nz; t += blockDim.x) {
        const int iz = t % L.Nz, w = t / L.Nz, iy = iy0 + w;
        if (iy >= L.Ny) continue;
        const int dip = L.cellmap[((size_t)ix * L.Ny + iy) * L.Nz + iz];
        if (dip < 0) continue;
        const int m = L.mat[dip];
        const C conv = invM * r[w * ls + iz];
        ys[dip] = cvt<C>(dg[m]) * xs[dip] - cvt<C>(cf[m]) * conv;
    }
}

// ---------------------------------------------------------------------------
// Generic pass along one axis of a batch of arrays [nb][n1][n2][n3].
// Reads the first in_len entries of every line (zero-extended to the FFT
// length), writes the first out_len outputs in place.
// ---------------------------------------------------------------------------
template <typename Rl, int W, bool INV, int AXIS>
__global__ void __launch_bounds__(FFT_THREADS) k_axis(cx<Rl>* data, int n1, int n2, int n3, int in_len, int out_len,
                                                      FftPlan p, const cx<Rl>* twg, const int* active, int per_sys) {
    using C = cx<Rl>;
    const int b = blockIdx.z;
    if (active && !active[b / per_sys]) return;
    const int Lf = p.L;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    for (int t = threadIdx.x; t < Lf; t += blockDim.x) tw[t] = twg[t];
    if (AXIS == 3) {
        const int ls = Lf + 1;
        C* A = tw + Lf;
        C* B = A + W * ls;
        const int i1 = blockIdx.y, i20 = blockIdx.x * W;
        C* base = data + ((size_t)b * n1 + i1) * (size_t)n2 * n3;
        for (int t = threadIdx.x; t < W * Lf; t += blockDim.x) {
            const int i = t % Lf, w = t / Lf, i2 = i20 + w;
            A[w * ls + i] = (i < in_len && i2 < n2) ? base[(size_t)i2 * n3 + i] : mk<C>(0.0, 0.0);
        }
        __syncthreads();
        const C* r = fft_lines<INV, false, W>(A, B, ls, 1, p, tw);
        for (int t = threadIdx.x; t < W * out_len; t += blockDim.x) {
            const int i = t % out_len, w = t / out_len, i2 = i20 + w;
            if (i2 < n2) base[(size_t)i2 * n3 + i] = r[w * ls + i];
        }
    } else {
        const int es = W + 1;
        C* A = tw + Lf;
        C* B = A + Lf * es;
        const int fixed = blockIdx.y, i30 = blockIdx.x * W;
        size_t base, stride;
        if (AXIS == 1) { base = (size_t)b * n1 * n2 * n3 + (size_t)fixed * n3; stride = (size_t)n2 * n3; }
        else { base = ((size_t)b * n1 + fixed) * (size_t)n2 * n3; stride = (size_t)n3; }
        C* d = data + base;
        for (int t = threadIdx.x; t < W * Lf; t += blockDim.x) {
            const int w = t % W, i = t / W, i3 = i30 + w;
            A[i * es + w] = (i < in_len && i3 < n3) ? d[(size_t)i * stride + i3] : mk<C>(0.0, 0.0);
        }
        __syncthreads();
        const C* r = fft_lines<INV, true, W>(A, B, 1, es, p, tw);
        for (int t = threadIdx.x; t < W * out_len; t += blockDim.x) {
            const int w = t % W, i = t / W, i3 = i30 + w;
            if (i3 < n3) d[(size_t)i * stride + i3] = r[i * es + w];
        }
    }
}

// ---------------------------------------------------------------------------
// Pass 3: forward x transform of the three components, product with the
// symmetric D-hat tensor, inverse x transform.  Block: W z-adjacent lines
// at fixed (s, ky); the 3W lines are interleaved in shared memory.
// ---------------------------------------------------------------------------
template <typename Rl, int W>
__global__ void __launch_bounds__(FFT_THREADS) k_xpass(LatticeDev L, MatvecArgs<Rl> a) {
    using C = cx<Rl>;
    const int s = blockIdx.z;
    if (a.active && !a.active[s]) return;
    const int ky = blockIdx.y, kz0 = blockIdx.x * W;
    const int Mx = L.Mx, Mz = L.Mz, Nx = L.Nx;
    constexpr int NL = 3 * W;
    constexpr int es = NL + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* A = tw + Mx;
    C* B = A + Mx * es;
    const C* twg = tw_of<Rl>(L, 0);
    for (int t = threadIdx.x; t < Mx; t += blockDim.x) tw[t] = twg[t];
    __syncthreads();
    const size_t plane = (size_t)L.Nx * Mz;
    C* U0 = a.U + ((size_t)s * 3 * L.My + ky) * plane;
    const size_t cstride = (size_t)L.My * plane;
    const C zero = mk<C>(0.0, 0.0);
    // forward x transforms of the 3W lines, read straight from U (rows ix >= Nx are zero)
    C* X = (L.px.nst % 2 == 0) ? B : A;   // the buffer the last forward stage does not read
    C* Y = (X == A) ? B : A;
    auto ld = [&](int l, int ix) -> C {
        const int c = l / W, kz = kz0 + l % W;
        return (ix < Nx && kz < Mz) ? U0[c * cstride + (size_t)ix * Mz + kz] : zero;
    };
    auto stX = [&](int l, int kx, C v) { X[kx * es + l] = v; };
    fft_lines_io<false, true, NL>(A, B, 1, es, L.px, tw, ld, stX);
    // D-hat product, in place in X
    const int hx = Mx / 2, hy = L.My / 2, hz = Mz / 2;
    const int kyr = ky <= hy ? ky : L.My - ky;
    const Rl sy = ky <= hy ? (Rl)1 : (Rl)-1;
    const size_t cs = (size_t)L.Hy * L.Hx * L.Hz;
    const C* Ds = a.Dr + (size_t)a.sys_slot[s] * 6 * cs;
    for (int t = threadIdx.x; t < W * Mx; t += blockDim.x) {
        const int w = t % W, kx = t / W, kz = kz0 + w;
        if (kz >= Mz) continue;
        const int kxr = kx <= hx ? kx : Mx - kx;
        const int kzr = kz <= hz ? kz : Mz - kz;
        const Rl sx = kx <= hx ? (Rl)1 : (Rl)-1;
        const Rl sz = kz <= hz ? (Rl)1 : (Rl)-1;
        const size_t idx = ((size_t)kyr * L.Hx + kxr) * L.Hz + kzr;
        const C dxx = Ds[idx], dxy = (sx * sy) * Ds[cs + idx], dxz = (sx * sz) * Ds[2 * cs + idx];
        const C dyy = Ds[3 * cs + idx], dyz = (sy * sz) * Ds[4 * cs + idx], dzz = Ds[5 * cs + idx];
        C* e = X + kx * es + w;
        const C Xv = e[0], Yv = e[W], Zv = e[2 * W];
        e[0] = dxx * Xv + dxy * Yv + dxz * Zv;
        e[W] = dxy * Xv + dyy * Yv + dyz * Zv;
        e[2 * W] = dxz * Xv + dyz * Yv + dzz * Zv;
    }
    __syncthreads();
    // inverse x transforms, the first Nx outputs written straight back to U
    auto ldX = [&](int l, int kx) -> C { return X[kx * es + l]; };
    auto st = [&](int l, int ix, C v) {
        const int c = l / W, kz = kz0 + l % W;
        if (ix < Nx && kz < Mz) U0[c * cstride + (size_t)ix * Mz + kz] = v;
    };
    fft_lines_io<true, true, NL>(Y, X, 1, es, L.px, tw, ldX, st);
}

// The x pass for the common lengths Mx = 64 (8 x 8) and Mx = 128 (8 x 8 x 2)
// with the stage descriptors known at compile time: the same shared-memory
// Stockham stages and D-hat product as k_xpass, but every index division,
// mask and loop bound folds to constants, and the block has one thread per
// radix-8 butterfly of a stage (3W lines x MX/8).
__host__ __device__ constexpr int cilog2(int v) { return (v > 0 && (v & (v - 1)) == 0) ? (v == 1 ? 0 : 1 + cilog2(v / 2)) : -1; }
__host__ __device__ constexpr FftStage cstage(int len, int r, int ns) {
    return FftStage{r, ns, cilog2(ns), len / r, cilog2(len / r), len / (ns * r)};
}

// First forward stage (sub-transform length 1, no twiddles) whose inputs
// j + r L/R lie in the zero padding for r >= R/2 when HALF (the lattice fills
// exactly the first half of the line): those inputs are compile-time zeros.
template <int R, int NL, int LEN, bool HALF, typename C, class In, class Out>
__device__ __forceinline__ void xstage_first(In in, Out out) {
    constexpr int nb = LEN / R;
    for (int t = threadIdx.x; t < NL * nb; t += blockDim.x) {
        const int line = t % NL, j = t / NL;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = (!HALF || r < R / 2) ? in(line, j + r * nb) : mk<C>(0.0, 0.0);
        Dft<R, false, C>::run(v);
#pragma unroll
        for (int r = 0; r < R; ++r) out(line, j * R + r, v[r]);
    }
}

// Last inverse stage (sub-transform length L/R, twiddle stride 1): with HALF
// only the outputs j + r L/R with r < R/2 (the lattice half) are formed.
template <int R, int NL, int LEN, bool HALF, typename C, class In, class Out>
__device__ __forceinline__ void xstage_last_inv(const C* __restrict__ tw, In in, Out out) {
    constexpr int nb = LEN / R;
    for (int t = threadIdx.x; t < NL * nb; t += blockDim.x) {
        const int line = t % NL, j = t / NL;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = in(line, j + r * nb);
#pragma unroll
        for (int r = 1; r < R; ++r) {
            C w = tw[r * j];
            w.y = -w.y;
            v[r] = v[r] * w;
        }
        Dft<R, true, C>::run(v);
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (!HALF || r < R / 2) out(line, j + r * nb, v[r]);
    }
}

template <int MX> struct XPlan;
template <> struct XPlan<64> { static constexpr int n = 2, r[3] = {8, 8, 1}; };
template <> struct XPlan<128> { static constexpr int n = 3, r[3] = {8, 8, 2}; };

template <typename Rl, int W, int MX, bool HALF>
__global__ void __launch_bounds__(3 * W * (MX / 8), (W == 16 && MX == 64 && sizeof(Rl) == 4) ? 4 : 1)
k_xpassc(LatticeDev L, MatvecArgs<Rl> a) {
    using C = cx<Rl>;
    using P = XPlan<MX>;
    constexpr int NT = 3 * W * (MX / 8);
    constexpr FftStage S0 = cstage(MX, P::r[0], 1);
    constexpr FftStage S1 = cstage(MX, P::r[1], P::r[0]);
    constexpr FftStage S2 = cstage(MX, P::n == 3 ? P::r[2] : 2, P::r[0] * P::r[1]);
    const int s = blockIdx.z;
    if (a.active && !a.active[s]) return;
    const int ky = blockIdx.y, kz0 = blockIdx.x * W;
    const int Mz = L.Mz, Nx = L.Nx;
    constexpr int NL = 3 * W;
    constexpr int es = NL + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* A = tw + MX;
    C* B = A + MX * es;
    const C* twg = tw_of<Rl>(L, 0);
    for (int t = threadIdx.x; t < MX; t += NT) tw[t] = twg[t];
    __syncthreads();
    const size_t plane = (size_t)Nx * Mz;
    C* U0 = a.U + ((size_t)s * 3 * L.My + ky) * plane;
    const size_t cstride = (size_t)L.My * plane;
    const C zero = mk<C>(0.0, 0.0);
    auto ld = [&](int l, int ix) -> C {
        const int c = l / W, kz = kz0 + l % W;
        return (ix < Nx && kz < Mz) ? U0[c * cstride + (size_t)ix * Mz + kz] : zero;
    };
    auto st = [&](int l, int ix, C v) {
        const int c = l / W, kz = kz0 + l % W;
        if (ix < Nx && kz < Mz) U0[c * cstride + (size_t)ix * Mz + kz] = v;
    };
    auto inA = [&](int l, int i) -> C { return A[i * es + l]; };
    auto inB = [&](int l, int i) -> C { return B[i * es + l]; };
    auto outA = [&](int l, int i, C v) { A[i * es + l] = v; };
    auto outB = [&](int l, int i, C v) { B[i * es + l] = v; };
    // forward x transforms of the 3W lines: U -> A -> B (-> A)
    xstage_first<P::r[0], NL, MX, HALF, C>(ld, outA);
    __syncthreads();
    fft_stage_f<P::r[1], false, true, NL>(S1, tw, inA, outB);
    __syncthreads();
    if (P::n == 3) {
        fft_stage_f<(P::n == 3 ? P::r[2] : 2), false, true, NL>(S2, tw, inB, outA);
        __syncthreads();
    }
    C* X = P::n == 3 ? A : B;         // holds the spectrum
    // D-hat product, in place
    const int hy = L.My / 2, hz = Mz / 2;
    const int kyr = ky <= hy ? ky : L.My - ky;
    const Rl sy = ky <= hy ? (Rl)1 : (Rl)-1;
    const size_t cs = (size_t)L.Hy * L.Hx * L.Hz;
    const C* Ds = a.Dr + (size_t)a.sys_slot[s] * 6 * cs + (size_t)kyr * L.Hx * L.Hz;
#pragma unroll 2
    for (int t = threadIdx.x; t < W * MX; t += NT) {
        const int w = t % W, kx = t / W, kz = kz0 + w;
        if (kz >= Mz) continue;
        const int kxr = kx <= MX / 2 ? kx : MX - kx;
        const int kzr = kz <= hz ? kz : Mz - kz;
        const Rl sx = kx <= MX / 2 ? (Rl)1 : (Rl)-1;
        const Rl sz = kz <= hz ? (Rl)1 : (Rl)-1;
        const C* d = Ds + (size_t)kxr * L.Hz + kzr;
        const C dxx = d[0], dxy = (sx * sy) * d[cs], dxz = (sx * sz) * d[2 * cs];
        const C dyy = d[3 * cs], dyz = (sy * sz) * d[4 * cs], dzz = d[5 * cs];
        C* e = X + kx * es + w;
        const C Xv = e[0], Yv = e[W], Zv = e[2 * W];
        e[0] = dxx * Xv + dxy * Yv + dxz * Zv;
        e[W] = dxy * Xv + dyy * Yv + dyz * Zv;
        e[2 * W] = dxz * Xv + dyz * Yv + dzz * Zv;
    }
    __syncthreads();
    // inverse x transforms back to U (first Nx outputs)
    if (P::n == 3) {
        fft_stage_f<P::r[0], true, true, NL>(S0, tw, inA, outB);
        __syncthreads();
        fft_stage_f<P::r[1], true, true, NL>(S1, tw, inB, outA);
        __syncthreads();
        xstage_last_inv<(P::n == 3 ? P::r[2] : 2), NL, MX, HALF, C>(tw, inA, st);
    } else {
        fft_stage_f<P::r[0], true, true, NL>(S0, tw, inB, outA);
        __syncthreads();
        xstage_last_inv<P::r[1], NL, MX, HALF, C>(tw, inA, st);
    }
}

// ---------------------------------------------------------------------------
// D-hat build: G~'(R) on the padded lattice, R in units of d, for n_slot
// wavenumbers kappa = k d.  Layout G[slot][comp][y][x][z].
//   G~' = exp(i kappa R)/R [kappa^2 (I - RR) - (1 - i kappa R)/R^2 (I - 3 RR)]   (Eq. 5)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int wrap_disp(int i, int n, int m, bool* ok) {
    if (i < n) return i;
    if (i > m - n) return i - m;
    *ok = false;
    return 0;
}

__global__ void k_green(LatticeDev L, const double2* kappa, double2* G) {
    const size_t M = (size_t)L.Mx * L.My * L.Mz;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= M) return;
    const int slot = blockIdx.y;
    const int z = (int)(idx % L.Mz);
    const int x = (int)((idx / L.Mz) % L.Mx);
    const int y = (int)(idx / ((size_t)L.Mz * L.Mx));
    bool ok = true;
    const double rx = wrap_disp(x, L.Nx, L.Mx, &ok);
    const double ry = wrap_disp(y, L.Ny, L.My, &ok);
    const double rz = wrap_disp(z, L.Nz, L.Mz, &ok);
    double2 g[6];
    for (int c = 0; c < 6; ++c) g[c] = make_double2(0.0, 0.0);
    const double rn2 = rx * rx + ry * ry + rz * rz;
    const bool near = L.igt && fabs(rx) <= IGT_NEAR && fabs(ry) <= IGT_NEAR && fabs(rz) <= IGT_NEAR;
    if (ok && rn2 > 0.0 && near) {
        // cell-averaged tensor to second order in kappa: exp(i kappa R)(-T0 + i kappa T1 + kappa^2 T2)
        const int side = 2 * IGT_NEAR + 1;
        const double* t = L.igt + ((size_t)(((int)rz + IGT_NEAR) * side + ((int)ry + IGT_NEAR)) * side +
                                   ((int)rx + IGT_NEAR)) * 18;
        const double rn = sqrt(rn2);
        const double2 kap = kappa[slot];
        double sn, cs;
        sincos(kap.x * rn, &sn, &cs);
        const double ex = exp(-kap.y * rn);
        const double2 ph = make_double2(ex * cs, ex * sn);
        const double2 ik = make_double2(-kap.y, kap.x);
        const double2 k2 = kap * kap;
        for (int c = 0; c < 6; ++c) {
            const double2 v = make_double2(-t[c], 0.0) + t[6 + c] * ik + t[12 + c] * k2;
            g[c] = ph * v;
        }
    } else if (ok && rn2 > 0.0) {
        const double rn = sqrt(rn2);
        const double h[3] = {rx / rn, ry / rn, rz / rn};
        const double2 kap = kappa[slot];
        // exp(i kappa R) / R
        const double2 ikr = make_double2(-kap.y * rn, kap.x * rn);
        double sn, cs;
        sincos(ikr.y, &sn, &cs);
        const double ex = exp(ikr.x) / rn;
        const double2 ph = make_double2(ex * cs, ex * sn);
        const double2 k2 = kap * kap;
        const double2 t = (1.0 / rn2) * make_double2(1.0 - ikr.x, -ikr.y);   // (1 - i kappa R)/R^2
        const int pa[6] = {0, 0, 0, 1, 1, 2}, pb[6] = {0, 1, 2, 1, 2, 2};
        for (int c = 0; c < 6; ++c) {
            const double hh = h[pa[c]] * h[pb[c]];
            const double dd = pa[c] == pb[c] ? 1.0 : 0.0;
            g[c] = ph * ((dd - hh) * k2 - (dd - 3.0 * hh) * t);
        }
    }
    double2* out = G + (size_t)slot * 6 * M + ((size_t)y * L.Mx + x) * L.Mz + z;
    for (int c = 0; c < 6; ++c) out[(size_t)c * M] = g[c];
}

__global__ void k_extract(LatticeDev L, int n_slot, const double2* G, double2* Dr64, float2* Dr32) {
    const size_t R = (size_t)L.Hx * L.Hy * L.Hz;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= R * 6 * n_slot) return;
    const size_t sc = idx / R;          // slot * 6 + comp
    const size_t r = idx % R;
    const int kz = (int)(r % L.Hz), kx = (int)((r / L.Hz) % L.Hx), ky = (int)(r / ((size_t)L.Hz * L.Hx));
    const size_t M = (size_t)L.Mx * L.My * L.Mz;
    const double2 v = G[sc * M + ((size_t)ky * L.Mx + kx) * L.Mz + kz];
    Dr64[idx] = v;
    Dr32[idx] = to_f(v);
}

// ---------------------------------------------------------------------------
// Fused slab passes (used when a slab fits shared memory): one block owns
// the x-slab ix of one (system, component).  Forward: gather the Ny x Nz
// corner, transform the Nz columns along y (CW at a time, into the slab
// buffer S[My][Nz]), then the My rows along z (CW at a time) and write the
// rows of U contiguously.  Inverse: the reverse order, then combine with x
// and scatter.  Dipoles are numbered slab-major (ix, iy, iz with iz
// fastest), so each slab's dipoles are contiguous and every global access
// is coalesced.  This turns the five passes into three.
// ---------------------------------------------------------------------------
// Row stride of the z-transform tile: runs of 8 elements of consecutive rows
// fall in disjoint bank groups when the stride is 8 mod 16.
__host__ __device__ __forceinline__ int slab_row_stride(int Mz) {
    int p = (Mz - 1) + ((Mz - 1) >> 3) + 1;   // padded row length (one slot per 8 elements)
    while (p % 16 != 8) ++p;
    return p;
}
// Slab buffer S[My][Nz]: rows padded to a multiple of 16 elements, and bit 3
// of the column index flipped on odd rows, so that the 8-element runs that
// consecutive rows read or write fall in disjoint banks without widening the
// rows.
__host__ __device__ __forceinline__ int slab_s_stride(int Nz) { return (Nz + 15) / 16 * 16; }
__device__ __forceinline__ int sidx(int y, int z, int sls) { return y * sls + (z ^ ((y & 1) << 3)); }

template <typename Rl, int CW>
__device__ __forceinline__ void slab_smem(unsigned char* raw, const LatticeDev& L, cx<Rl>*& twy, cx<Rl>*& twz,
                                          cx<Rl>*& S, cx<Rl>*& A, cx<Rl>*& B) {
    using C = cx<Rl>;
    const int scr = max(L.My * (CW + 1), CW * slab_row_stride(L.Mz));
    twy = reinterpret_cast<C*>(raw);
    twz = twy + L.My;
    S = twz + L.Mz;
    A = S + L.My * slab_s_stride(L.Nz);
    B = A + scr;
    const C* gy = tw_of<Rl>(L, 1);
    const C* gz = tw_of<Rl>(L, 2);
    for (int t = threadIdx.x; t < L.My; t += blockDim.x) twy[t] = gy[t];
    for (int t = threadIdx.x; t < L.Mz; t += blockDim.x) twz[t] = gz[t];
}

template <typename Rl, int CW>
__global__ void __launch_bounds__(FFT_THREADS) k_slab_fwd(LatticeDev L, MatvecArgs<Rl> a) {
    using C = cx<Rl>;
    const int ix = blockIdx.x, b = blockIdx.y, s = b / 3, c = b % 3;
    if (a.active && !a.active[s]) return;
    const int My = L.My, Ny = L.Ny, Nz = L.Nz;
    const int sls = slab_s_stride(Nz), es = CW + 1, rls = slab_row_stride(L.Mz);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *twy, *twz, *S, *A, *B;
    slab_smem<Rl, CW>(smem_raw, L, twy, twz, S, A, B);
    __syncthreads();
    const C* xs = a.x + ((size_t)s * 3 + c) * L.N;
    const double2* cf = a.coef + (size_t)s * EELS_MAX_MAT;
    const int* cm = L.cellmap + (size_t)ix * Ny * Nz;
    const C zero = mk<C>(0.0, 0.0);
    // y transforms of the Nz columns (CW at a time): gathered from x, into S
    for (int iz0 = 0; iz0 < Nz; iz0 += CW) {
        auto ld = [&](int l, int y) -> C {
            const int iz = iz0 + l;
            if (y >= Ny || iz >= Nz) return zero;
            const int dip = cm[y * Nz + iz];
            return dip >= 0 ? xs[dip] * cvt<C>(cf[L.mat[dip]]) : zero;
        };
        auto st = [&](int l, int y, C v) {
            const int iz = iz0 + l;
            if (iz < Nz) S[sidx(y, iz, sls)] = v;
        };
        fft_lines_io<false, true, CW>(A, B, 1, es, L.py, twy, ld, st);
    }
    // z transforms of the My rows (CW at a time): from S, rows written to U
    C* U = a.U + (((size_t)s * 3 + c) * My * L.Nx + ix) * L.Mz;
    const size_t row = (size_t)L.Nx * L.Mz;
    for (int ky0 = 0; ky0 < My; ky0 += CW) {
        auto ld = [&](int l, int z) -> C {
            const int ky = ky0 + l;
            return (z < Nz && ky < My) ? S[sidx(ky, z, sls)] : zero;
        };
        auto st = [&](int l, int z, C v) {
            const int ky = ky0 + l;
            if (ky < My) U[(size_t)ky * row + z] = v;
        };
        fft_lines_io<false, false, CW, true>(A, B, rls, 1, L.pz, twz, ld, st);
    }
}

template <typename Rl, int CW>
__global__ void __launch_bounds__(FFT_THREADS) k_slab_inv(LatticeDev L, MatvecArgs<Rl> a, Rl invM) {
    using C = cx<Rl>;
    const int ix = blockIdx.x, b = blockIdx.y, s = b / 3, c = b % 3;
    if (a.active && !a.active[s]) return;
    const int My = L.My, Ny = L.Ny, Nz = L.Nz;
    const int sls = slab_s_stride(Nz), es = CW + 1, rls = slab_row_stride(L.Mz);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *twy, *twz, *S, *A, *B;
    slab_smem<Rl, CW>(smem_raw, L, twy, twz, S, A, B);
    __syncthreads();
    const C zero = mk<C>(0.0, 0.0);
    // inverse z transforms of the My rows of U (CW at a time), first Nz outputs into S
    const C* U = a.U + (((size_t)s * 3 + c) * My * L.Nx + ix) * L.Mz;
    const size_t row = (size_t)L.Nx * L.Mz;
    for (int ky0 = 0; ky0 < My; ky0 += CW) {
        auto ld = [&](int l, int z) -> C {
            const int ky = ky0 + l;
            return ky < My ? U[(size_t)ky * row + z] : zero;
        };
        auto st = [&](int l, int z, C v) {
            const int ky = ky0 + l;
            if (ky < My && z < Nz) S[sidx(ky, z, sls)] = v;
        };
        fft_lines_io<true, false, CW, true>(A, B, rls, 1, L.pz, twz, ld, st);
    }
    // inverse y transforms of the Nz columns, first Ny outputs combined with x and scattered
    const C* xs = a.x + ((size_t)s * 3 + c) * L.N;
    C* ys = a.y + ((size_t)s * 3 + c) * L.N;
    const double2* cf = a.coef + (size_t)s * EELS_MAX_MAT;
    const double2* dg = a.diag + (size_t)s * EELS_MAX_MAT;
    const int* cm = L.cellmap + (size_t)ix * Ny * Nz;
    Rl dot[2] = {0, 0};
    for (int iz0 = 0; iz0 < Nz; iz0 += CW) {
        auto ld = [&](int l, int y) -> C {
            const int iz = iz0 + l;
            return iz < Nz ? S[sidx(y, iz, sls)] : zero;
        };
        auto st = [&](int l, int y, C v) {
            const int iz = iz0 + l;
            if (y >= Ny || iz >= Nz) return;
            const int dip = cm[y * Nz + iz];
            if (dip < 0) return;
            const int m = L.mat[dip];
            const C xv = xs[dip];
            const C yv = cvt<C>(dg[m]) * xv - cvt<C>(cf[m]) * (invM * v);
            ys[dip] = yv;
            dot[0] += xv.x * yv.x - xv.y * yv.y;
            dot[1] += xv.x * yv.y + xv.y * yv.x;
        };
        fft_lines_io<true, true, CW>(A, B, 1, es, L.py, twy, ld, st);
    }
    if (a.dot_part) {
        // block sum in a fixed order (warp shuffles, then thread 0 over the warps)
        for (int o = 16; o > 0; o >>= 1) {
            dot[0] += __shfl_xor_sync(0xffffffffu, dot[0], o);
            dot[1] += __shfl_xor_sync(0xffffffffu, dot[1], o);
        }
        Rl* red = reinterpret_cast<Rl*>(A);
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        if (lane == 0) { red[2 * wid] = dot[0]; red[2 * wid + 1] = dot[1]; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double s0 = 0, s1 = 0;
            for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { s0 += red[2 * i]; s1 += red[2 * i + 1]; }
            double* p = a.dot_part + (((size_t)s * 3 + c) * L.Nx + ix) * 4;
            p[0] = s0; p[1] = s1; p[2] = 0.0; p[3] = 0.0;
        }
    }
}

// ---------------------------------------------------------------------------
// Fused slab passes for My = Mz = L = 64 or 128 in FP32, register resident.
//
// A warp transforms 4 lines at once (fft_warp.cuh): lane = q + 4p holds, for
// its line q, the elements p + 8r (r < R = L/8) of the line, and the
// transform leaves element j + 8m in register m of lane j.  Between the y and
// the z transforms the slab S[L][Nz] sits in shared memory (row stride
// 4 mod 16: the 4 x 4 (line, lane) patterns of every access hit distinct
// banks); the block synchronises once per pass.  Every loop over line quads
// loads the next quad's inputs before transforming the current one, so the
// global loads of one quad overlap the arithmetic of the previous one.
// HALF: Ny = Nz = L/2 (the lattice fills exactly half of every line): the
// zero padding and the discarded outputs are known at compile time.  FAST:
// every column's occupied cells are contiguous in z, so a dipole's index is
// the column's base plus iz (no cell-map load).
// ---------------------------------------------------------------------------
// Dipole at depth iz of a column whose occupied cells are contiguous:
// ci = (index of the column's first dipole - its first iz, first iz, last iz + 1).
__device__ __forceinline__ int col_dip(int4 ci, int iz) { return (iz >= ci.y && iz < ci.z) ? ci.x + iz : -1; }

template <int R> struct SlabR {
    static constexpr int L = 8 * R;
    static constexpr int SLS = R == 8 ? 36 : 68;           // slab row stride
    static constexpr int TILE = R == 8 ? R64_TILE : R128_TILE;
};

template <int R> struct SlabRSmem {
    float2 tw2[(R - 1) * 8];                     // exp(-2 pi i p k / L) at [k - 1][p]: conflict-free per k
    float2 cf[EELS_MAX_MAT], dg[EELS_MAX_MAT];   // this system's per-material coefficients
    float2 S[SlabR<R>::L * SlabR<R>::SLS];
    float2 tile[FFT_THREADS / 32][SlabR<R>::TILE];
    int4 ci[SlabR<R>::L / 2];                    // this slab's column table (contiguous columns)
};

// Persistent forward slab pass: the grid holds as many blocks as fit on the
// GPU at once, and each block walks the (system, component, slab) items with
// a stride of the grid size.  For single-material lattices with contiguous
// columns, a block loads the first column quad of its next item while it runs
// the z transforms of the current one, so the gather's latency is hidden
// behind arithmetic instead of opening every item.
template <int R, bool HALF, bool FAST>
__global__ void __launch_bounds__(FFT_THREADS, R == 8 ? 4 : 2) k_slab_fwd_r(LatticeDev L, MatvecArgs<float> a) {
    using C = float2;
    using P = SlabR<R>;
    constexpr int LEN = P::L, SLS = P::SLS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SlabRSmem<R>& sm = *reinterpret_cast<SlabRSmem<R>*>(smem_raw);
    const int Ny = L.Ny, Nz = L.Nz, Nx = L.Nx, warp = threadIdx.x >> 5, lane = threadIdx.x & 31, q = lane & 3,
              p = lane >> 2;
    const int nwarp = blockDim.x >> 5;
    const int n_items = a.S * 3 * Nx;
    const bool one_mat = L.nmat == 1;
    const bool prefetch = FAST && one_mat;
    const float2* twg = tw_of<float>(L, 1);          // My = Mz: the y and z tables coincide
    for (int t = threadIdx.x; t < (R - 1) * 8; t += blockDim.x) sm.tw2[t] = twg[(t & 7) * ((t >> 3) + 1)];
    float2* tile = sm.tile[warp];
    auto tw = [&](int k) { return sm.tw2[(k - 1) * 8 + p]; };
    const C zero = make_float2(0.f, 0.f);
    const int stride = nwarp * 4;
    auto active = [&](int item) { return !a.active || a.active[item / (3 * Nx)]; };
    auto next_item = [&](int item) {
        for (item += gridDim.x; item < n_items && !active(item); item += gridDim.x) {}
        return item;
    };
    // raw x values of the first column quad (iz0 = 4 warp) of an item, dipoles
    // addressed through the column table in global memory
    auto gather_raw = [&](int item, C (&v)[R]) {
        const int s = item / (3 * Nx), c = (item / Nx) % 3, ix = item % Nx, iz = warp * 4 + q;
        const C* xs = a.x + ((size_t)s * 3 + c) * L.N;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int y = p + 8 * r;
            v[r] = zero;
            if ((HALF ? r < R / 2 : y < Ny) && iz < Nz) {
                const int dip = col_dip(L.colinfo[(size_t)ix * Ny + y], iz);
                if (dip >= 0) v[r] = xs[dip];
            }
        }
    };
    C pf[R];
    int item = blockIdx.x;
    if (item < n_items && !active(item)) item = next_item(item);
    if (prefetch && item < n_items && warp * 4 < Nz) gather_raw(item, pf);
    for (; item < n_items;) {
        const int s = item / (3 * Nx), c = (item / Nx) % 3, ix = item % Nx;
        if (threadIdx.x < EELS_MAX_MAT) sm.cf[threadIdx.x] = to_f(a.coef[(size_t)s * EELS_MAX_MAT + threadIdx.x]);
        if (FAST)
            for (int t = threadIdx.x; t < Ny; t += blockDim.x) sm.ci[t] = L.colinfo[(size_t)ix * Ny + t];
        __syncthreads();
        const C* xs = a.x + ((size_t)s * 3 + c) * L.N;
        const int* cm = L.cellmap + (size_t)ix * Ny * Nz;
        // y transforms of the Nz columns, 4 per warp: gathered from x, into S
        auto gather = [&](int iz0, C (&v)[R]) {
            const int iz = iz0 + q;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int y = p + 8 * r;
                v[r] = zero;
                if ((HALF ? r < R / 2 : y < Ny) && iz < Nz) {
                    const int dip = FAST ? col_dip(sm.ci[y], iz) : cm[y * Nz + iz];
                    if (dip >= 0) v[r] = xs[dip] * (one_mat ? sm.cf[0] : sm.cf[L.mat[dip]]);
                }
            }
        };
        C vn[R];
        if (warp * 4 < Nz) {
            if (prefetch) {
#pragma unroll
                for (int r = 0; r < R; ++r) vn[r] = pf[r] * sm.cf[0];
            } else {
                gather(warp * 4, vn);
            }
        }
        for (int iz0 = warp * 4; iz0 < Nz; iz0 += stride) {
            C v[R];
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = vn[r];
            if (iz0 + stride < Nz) gather(iz0 + stride, vn);
            fft_warp_t<R, false, HALF>(v, tile, q, p, tw);
            const int iz = iz0 + q;
            if (iz < Nz) {
#pragma unroll
                for (int m = 0; m < R; ++m) sm.S[(p + 8 * m) * SLS + iz] = v[m];
            }
        }
        __syncthreads();
        const int nxt = next_item(item);
        if (prefetch && nxt < n_items && warp * 4 < Nz) gather_raw(nxt, pf);
        // z transforms of the LEN rows, 4 per warp: from S, written to U
        C* U = a.U + (((size_t)s * 3 + c) * LEN * L.Nx + ix) * LEN;
        const size_t row = (size_t)L.Nx * LEN;
        for (int ky0 = warp * 4; ky0 < LEN; ky0 += stride) {
            const int ky = ky0 + q;
            C v[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int z = p + 8 * r;
                v[r] = (HALF ? r < R / 2 : z < Nz) ? sm.S[ky * SLS + z] : zero;
            }
            fft_warp_t<R, false, HALF>(v, tile, q, p, tw);
#pragma unroll
            for (int m = 0; m < R; ++m) U[(size_t)ky * row + p + 8 * m] = v[m];
        }
        item = nxt;
        __syncthreads();                              // S, ci and cf are refilled for the next item
    }
}

template <int R, bool HALF, bool FAST>
__global__ void __launch_bounds__(FFT_THREADS, R == 8 ? 4 : 2) k_slab_inv_r(LatticeDev L, MatvecArgs<float> a, float invM) {
    using C = float2;
    using P = SlabR<R>;
    constexpr int LEN = P::L, SLS = P::SLS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SlabRSmem<R>& sm = *reinterpret_cast<SlabRSmem<R>*>(smem_raw);
    __shared__ float red[2 * FFT_THREADS / 32];
    const int ix = blockIdx.x, b = blockIdx.y, s = b / 3, c = b % 3;
    if (a.active && !a.active[s]) return;
    const int Ny = L.Ny, Nz = L.Nz, warp = threadIdx.x >> 5, lane = threadIdx.x & 31, q = lane & 3, p = lane >> 2;
    const int nwarp = blockDim.x >> 5;
    const float2* twg = tw_of<float>(L, 2);
    for (int t = threadIdx.x; t < (R - 1) * 8; t += blockDim.x) sm.tw2[t] = twg[(t & 7) * ((t >> 3) + 1)];
    if (threadIdx.x < EELS_MAX_MAT) {
        sm.cf[threadIdx.x] = to_f(a.coef[(size_t)s * EELS_MAX_MAT + threadIdx.x]);
        sm.dg[threadIdx.x] = to_f(a.diag[(size_t)s * EELS_MAX_MAT + threadIdx.x]);
    }
    if (FAST)
        for (int t = threadIdx.x; t < Ny; t += blockDim.x) sm.ci[t] = L.colinfo[(size_t)ix * Ny + t];
    const bool one_mat = L.nmat == 1;
    __syncthreads();
    float2* tile = sm.tile[warp];
    auto tw = [&](int k) { return sm.tw2[(k - 1) * 8 + p]; };
    const int stride = nwarp * 4;
    // inverse z transforms of the LEN rows of U, first Nz outputs into S
    const C* U = a.U + (((size_t)s * 3 + c) * LEN * L.Nx + ix) * LEN;
    const size_t row = (size_t)L.Nx * LEN;
    C vn[R];
#pragma unroll
    for (int r = 0; r < R; ++r) vn[r] = U[(size_t)(warp * 4 + q) * row + p + 8 * r];
    for (int ky0 = warp * 4; ky0 < LEN; ky0 += stride) {
        const int ky = ky0 + q;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = vn[r];
        if (ky0 + stride < LEN) {
#pragma unroll
            for (int r = 0; r < R; ++r) vn[r] = U[(size_t)(ky + stride) * row + p + 8 * r];
        }
        fft_warp_t<R, true, false>(v, tile, q, p, tw);
#pragma unroll
        for (int m = 0; m < R; ++m) {
            const int z = p + 8 * m;
            if (HALF ? m < R / 2 : z < Nz) sm.S[ky * SLS + z] = v[m];
        }
    }
    __syncthreads();
    // inverse y transforms of the Nz columns, first Ny outputs combined with x
    // and scattered; each lane loads its x values before its transform
    const C* xs = a.x + ((size_t)s * 3 + c) * L.N;
    C* ys = a.y + ((size_t)s * 3 + c) * L.N;
    const int* cm = L.cellmap + (size_t)ix * Ny * Nz;
    constexpr int RO = HALF ? R / 2 : R;             // registers that can hold lattice rows
    float dot0 = 0.f, dot1 = 0.f;
    for (int iz0 = warp * 4; iz0 < Nz; iz0 += stride) {
        const int iz = iz0 + q;
        int dip[RO];
        C xv[RO];
#pragma unroll
        for (int m = 0; m < RO; ++m) {
            const int y = p + 8 * m;
            dip[m] = -1;
            if (iz < Nz && (HALF || y < Ny)) dip[m] = FAST ? col_dip(sm.ci[y], iz) : cm[y * Nz + iz];
            xv[m] = dip[m] >= 0 ? xs[dip[m]] : make_float2(0.f, 0.f);
        }
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = iz < Nz ? sm.S[(p + 8 * r) * SLS + iz] : make_float2(0.f, 0.f);
        fft_warp_t<R, true, false>(v, tile, q, p, tw);
#pragma unroll
        for (int m = 0; m < RO; ++m) {
            if (dip[m] < 0) continue;
            const int mt = one_mat ? 0 : L.mat[dip[m]];
            const C yv = sm.dg[mt] * xv[m] - sm.cf[mt] * (invM * v[m]);
            ys[dip[m]] = yv;
            dot0 += xv[m].x * yv.x - xv[m].y * yv.y;
            dot1 += xv[m].x * yv.y + xv[m].y * yv.x;
        }
    }
    if (a.dot_part) {
        // block sum in a fixed order (warp shuffles, then thread 0 over the warps)
        for (int o = 16; o > 0; o >>= 1) {
            dot0 += __shfl_xor_sync(0xffffffffu, dot0, o);
            dot1 += __shfl_xor_sync(0xffffffffu, dot1, o);
        }
        if (lane == 0) { red[2 * warp] = dot0; red[2 * warp + 1] = dot1; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double s0 = 0, s1 = 0;
            for (int i = 0; i < nwarp; ++i) { s0 += red[2 * i]; s1 += red[2 * i + 1]; }
            double* pp = a.dot_part + (((size_t)s * 3 + c) * L.Nx + ix) * 4;
            pp[0] = s0; pp[1] = s1; pp[2] = 0.0; pp[3] = 0.0;
        }
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
static const size_t kSmemCap = 220 * 1024;

template <typename Rl> static size_t smem_zpass(const LatticeDev& L, int W) { return (size_t)(L.Mz + 2 * W * (L.Mz + 1)) * sizeof(cx<Rl>); }
template <typename Rl> static size_t smem_xpass(const LatticeDev& L, int W) { return (size_t)(L.Mx + 2 * L.Mx * (3 * W + 1)) * sizeof(cx<Rl>); }
template <typename Rl> static size_t smem_axis(int Lf, int W, int axis) {
    return axis == 3 ? (size_t)(Lf + 2 * W * (Lf + 1)) * sizeof(cx<Rl>) : (size_t)(Lf + 2 * Lf * (W + 1)) * sizeof(cx<Rl>);
}

template <typename K> static void allow_smem(K kernel) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap);
    // these kernels keep their working tiles in shared memory: give it the whole carveout
    cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
}

// Pick the widest tile whose shared memory fits a budget that leaves room
// for two resident blocks per SM (falling back to one block per SM).
template <typename F> static int pick_w(F smem_of) {
    for (int W : {32, 16, 8})
        if (smem_of(W) <= 110 * 1024) return W;
    for (int W : {16, 8})
        if (smem_of(W) <= kSmemCap) return W;
    return 0;
}

template <typename Rl, int W, bool INV, int AXIS>
static void axis_launch_w(cx<Rl>* data, int nb, int n1, int n2, int n3, int in_len, int out_len, const FftPlan& p,
                          const cx<Rl>* tw, const int* active, int per_sys, cudaStream_t st) {
    dim3 grid;
    if (AXIS == 3) grid = dim3((n2 + W - 1) / W, n1, nb);
    else if (AXIS == 1) grid = dim3((n3 + W - 1) / W, n2, nb);
    else grid = dim3((n3 + W - 1) / W, n1, nb);
    count_launch();
    k_axis<Rl, W, INV, AXIS><<<grid, FFT_THREADS, smem_axis<Rl>(p.L, W, AXIS), st>>>(data, n1, n2, n3, in_len, out_len, p, tw,
                                                                                    active, per_sys);
}

template <typename Rl, bool INV, int AXIS>
static void axis_launch(cx<Rl>* data, int nb, int n1, int n2, int n3, int in_len, int out_len, const FftPlan& p,
                        const cx<Rl>* tw, const int* active, int per_sys, cudaStream_t st) {
    const int W = pick_w([&](int w) { return smem_axis<Rl>(p.L, w, AXIS); });
    if (W == 32) axis_launch_w<Rl, 32, INV, AXIS>(data, nb, n1, n2, n3, in_len, out_len, p, tw, active, per_sys, st);
    else if (W == 16) axis_launch_w<Rl, 16, INV, AXIS>(data, nb, n1, n2, n3, in_len, out_len, p, tw, active, per_sys, st);
    else axis_launch_w<Rl, 8, INV, AXIS>(data, nb, n1, n2, n3, in_len, out_len, p, tw, active, per_sys, st);
}

template <typename Rl> static const cx<Rl>* host_tw(const LatticeDev& L, int axis);
template <> const double2* host_tw<double>(const LatticeDev& L, int axis) { return axis == 0 ? L.tw64x : (axis == 1 ? L.tw64y : L.tw64z); }
template <> const float2* host_tw<float>(const LatticeDev& L, int axis) { return axis == 0 ? L.tw32x : (axis == 1 ? L.tw32y : L.tw32z); }

template <typename Rl, int W>
static void zpass_launch(const LatticeDev& L, const MatvecArgs<Rl>& a, bool inv, cudaStream_t st) {
    dim3 grid((L.Ny + W - 1) / W, L.Nx, a.S * 3);
    const size_t sm = smem_zpass<Rl>(L, W);
    count_launch();
    if (!inv) k_zfwd<Rl, W><<<grid, FFT_THREADS, sm, st>>>(L, a);
    else k_zinv<Rl, W><<<grid, FFT_THREADS, sm, st>>>(L, a, (Rl)(1.0 / ((double)L.Mx * L.My * L.Mz)));
}

template <typename Rl, int W>
static void xpass_launch(const LatticeDev& L, const MatvecArgs<Rl>& a, cudaStream_t st) {
    dim3 grid((L.Mz + W - 1) / W, L.My, a.S);
    count_launch();
    const auto& px = L.px;
    const bool x64 = L.Mx == 64 && px.nst == 2 && px.st[0].R == 8 && px.st[1].R == 8;
    const bool x128 = L.Mx == 128 && px.nst == 3 && px.st[0].R == 8 && px.st[1].R == 8 && px.st[2].R == 2;
    const bool half = 2 * L.Nx == L.Mx;             // the lattice fills exactly half of each line
    if (x64) {
        if (half) k_xpassc<Rl, W, 64, true><<<grid, 3 * W * 8, smem_xpass<Rl>(L, W), st>>>(L, a);
        else k_xpassc<Rl, W, 64, false><<<grid, 3 * W * 8, smem_xpass<Rl>(L, W), st>>>(L, a);
        return;
    }
    if constexpr (W <= 16) {                         // 3W x 16 threads per block
        if (x128) {
            if (half) k_xpassc<Rl, W, 128, true><<<grid, 3 * W * 16, smem_xpass<Rl>(L, W), st>>>(L, a);
            else k_xpassc<Rl, W, 128, false><<<grid, 3 * W * 16, smem_xpass<Rl>(L, W), st>>>(L, a);
            return;
        }
    }
    k_xpass<Rl, W><<<grid, FFT_THREADS, smem_xpass<Rl>(L, W), st>>>(L, a);
}

template <typename Rl, int CW> static size_t smem_slab(const LatticeDev& L) {
    const size_t scr = (size_t)std::max(L.My * (CW + 1), CW * slab_row_stride(L.Mz));
    return ((size_t)L.My + L.Mz + (size_t)L.My * slab_s_stride(L.Nz) + 2 * scr) * sizeof(cx<Rl>);
}

// Widest column tile whose fused-slab shared memory fits one block (0: none).
template <typename Rl> static int pick_slab(const LatticeDev& L) {
    if (smem_slab<Rl, 32>(L) <= 110 * 1024) return 32;
    if (smem_slab<Rl, 16>(L) <= 110 * 1024) return 16;
    if (smem_slab<Rl, 16>(L) <= kSmemCap) return 16;
    if (smem_slab<Rl, 8>(L) <= kSmemCap) return 8;
    return 0;
}

template <typename Rl, int CW>
static void slab_launch(const LatticeDev& L, const MatvecArgs<Rl>& a, bool inv, cudaStream_t st) {
    dim3 grid(L.Nx, a.S * 3);
    const size_t sm = smem_slab<Rl, CW>(L);
    count_launch();
    if (!inv) k_slab_fwd<Rl, CW><<<grid, FFT_THREADS, sm, st>>>(L, a);
    else k_slab_inv<Rl, CW><<<grid, FFT_THREADS, sm, st>>>(L, a, (Rl)(1.0 / ((double)L.Mx * L.My * L.Mz)));
}

// Register-resident slab kernels: FP32 with 64- or 128-point y and z transforms.
// Multiprocessors of the current device (queried once per device).
static int sm_count() {
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) { cudaGetLastError(); return 132; }
    if (!cache[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
            cudaGetLastError();
            n = 132;
        }
        cache[dev] = n;
    }
    return cache[dev];
}

template <int R, bool HALF, bool FAST>
static void slab_r_launch(const LatticeDev& L, const MatvecArgs<float>& a, bool inv, cudaStream_t st) {
    const size_t sm = sizeof(SlabRSmem<R>);
    const float invM = (float)(1.0 / ((double)L.Mx * L.My * L.Mz));
    if (!inv) {
        // persistent: the blocks resident at once (2 or 4 per multiprocessor)
        const int items = a.S * 3 * L.Nx;
        const int blocks = std::min(items, sm_count() * (R == 8 ? 4 : 2));
        k_slab_fwd_r<R, HALF, FAST><<<blocks, FFT_THREADS, sm, st>>>(L, a);
    } else {
        k_slab_inv_r<R, HALF, FAST><<<dim3(L.Nx, a.S * 3), FFT_THREADS, sm, st>>>(L, a, invM);
    }
}

template <int R>
static void slab_r_any(const LatticeDev& L, const MatvecArgs<float>& a, bool inv, cudaStream_t st) {
    const bool half = 2 * L.Ny == 8 * R && 2 * L.Nz == 8 * R;
    count_launch();
    if (half && L.contig) slab_r_launch<R, true, true>(L, a, inv, st);
    else if (half) slab_r_launch<R, true, false>(L, a, inv, st);
    else if (L.contig) slab_r_launch<R, false, true>(L, a, inv, st);
    else slab_r_launch<R, false, false>(L, a, inv, st);
}

template <typename Rl> static bool slab_reg_launch(const LatticeDev& L, const MatvecArgs<Rl>& a, bool inv, cudaStream_t st);
template <> bool slab_reg_launch<double>(const LatticeDev&, const MatvecArgs<double>&, bool, cudaStream_t) { return false; }
template <> bool slab_reg_launch<float>(const LatticeDev& L, const MatvecArgs<float>& a, bool inv, cudaStream_t st) {
    if (L.My == 64 && L.Mz == 64) { slab_r_any<8>(L, a, inv, st); return true; }
    if (L.My == 128 && L.Mz == 128) { slab_r_any<16>(L, a, inv, st); return true; }
    return false;
}

template <typename Rl> static void slab_launch_any(const LatticeDev& L, const MatvecArgs<Rl>& a, bool inv, int cw,
                                                   cudaStream_t st) {
    if (slab_reg_launch<Rl>(L, a, inv, st)) return;
    if (cw == 32) slab_launch<Rl, 32>(L, a, inv, st);
    else if (cw == 16) slab_launch<Rl, 16>(L, a, inv, st);
    else slab_launch<Rl, 8>(L, a, inv, st);
}

// Widest x-pass tile (W lines per component) whose two buffers fit a
// quarter of an SM's shared memory, so that four blocks are resident.
template <typename Rl> static int pick_xpass_w(const LatticeDev& L) {
    for (int W : {32, 16, 8})
        if (smem_xpass<Rl>(L, W) <= 56 * 1024) return W;
    return pick_w([&](int w) { return smem_xpass<Rl>(L, w); });
}

template <typename Rl> static int tuned_w(const LatticeDev& L) { return sizeof(Rl) == 4 ? L.xw32 : L.xw64; }

template <typename Rl> static void xpass_w(const LatticeDev& L, const MatvecArgs<Rl>& a, int wx, cudaStream_t st) {
    if (wx == 32) xpass_launch<Rl, 32>(L, a, st);
    else if (wx == 16) xpass_launch<Rl, 16>(L, a, st);
    else xpass_launch<Rl, 8>(L, a, st);
}

template <typename Rl>
int autotune_xpass(const LatticeDev& L, const MatvecArgs<Rl>& a, cudaStream_t st) {
    int best = pick_xpass_w<Rl>(L);
    float best_ms = 0.f;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return best;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return best; }
    bool first = true;
    for (int w : {8, 16, 32}) {
        if (smem_xpass<Rl>(L, w) > kSmemCap) continue;
        xpass_w<Rl>(L, a, w, st);                   // warm-up
        cudaEventRecord(e0, st);
        for (int r = 0; r < 3; ++r) xpass_w<Rl>(L, a, w, st);
        cudaEventRecord(e1, st);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) break;
        if (first || ms < best_ms) { best = w; best_ms = ms; first = false; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}
template int autotune_xpass<float>(const LatticeDev&, const MatvecArgs<float>&, cudaStream_t);
template int autotune_xpass<double>(const LatticeDev&, const MatvecArgs<double>&, cudaStream_t);

template <typename Rl> static void xpass_any(const LatticeDev& L, const MatvecArgs<Rl>& a, cudaStream_t st) {
    if constexpr (sizeof(Rl) == 4) {
        if (launch_xpass_reg(L, a, st)) return;
    }
    const int wx = tuned_w<Rl>(L) ? tuned_w<Rl>(L) : pick_xpass_w<Rl>(L);
    if (wx == 32) xpass_launch<Rl, 32>(L, a, st);
    else if (wx == 16) xpass_launch<Rl, 16>(L, a, st);
    else xpass_launch<Rl, 8>(L, a, st);
}

template <typename Rl>
bool launch_matvec(const LatticeDev& L, const MatvecArgs<Rl>& a, cudaStream_t st) {
    const int cw = pick_slab<Rl>(L);
    if (cw) {   // three passes: slab (gather, y, z) -> x * D-hat * x -> slab (z, y, scatter)
        slab_launch_any<Rl>(L, a, false, cw, st);
        xpass_any<Rl>(L, a, st);
        slab_launch_any<Rl>(L, a, true, cw, st);
        return a.dot_part != nullptr;
    }
    const int wz = pick_w([&](int w) { return smem_zpass<Rl>(L, w); });
    if (wz == 32) zpass_launch<Rl, 32>(L, a, false, st);
    else if (wz == 16) zpass_launch<Rl, 16>(L, a, false, st);
    else zpass_launch<Rl, 8>(L, a, false, st);
    axis_launch<Rl, false, 1>(a.U, a.S * 3, L.My, L.Nx, L.Mz, L.Ny, L.My, L.py, host_tw<Rl>(L, 1), a.active, 3, st);
    xpass_any<Rl>(L, a, st);
    axis_launch<Rl, true, 1>(a.U, a.S * 3, L.My, L.Nx, L.Mz, L.My, L.Ny, L.py, host_tw<Rl>(L, 1), a.active, 3, st);
    if (wz == 32) zpass_launch<Rl, 32>(L, a, true, st);
    else if (wz == 16) zpass_launch<Rl, 16>(L, a, true, st);
    else zpass_launch<Rl, 8>(L, a, true, st);
    return false;
}

template <typename Rl, int W> static void prepare_w() {
    allow_smem(k_zfwd<Rl, W>);
    allow_smem(k_zinv<Rl, W>);
    allow_smem(k_xpass<Rl, W>);
    allow_smem(k_xpassc<Rl, W, 64, true>);
    allow_smem(k_xpassc<Rl, W, 64, false>);
    if constexpr (W <= 16) {
        allow_smem(k_xpassc<Rl, W, 128, true>);
        allow_smem(k_xpassc<Rl, W, 128, false>);
    }
    allow_smem(k_axis<Rl, W, false, 1>);
    allow_smem(k_axis<Rl, W, true, 1>);
    allow_smem(k_axis<Rl, W, false, 2>);
    allow_smem(k_axis<Rl, W, false, 3>);
    allow_smem(k_slab_fwd<Rl, W>);
    allow_smem(k_slab_inv<Rl, W>);
}

void prepare_far_kernels();
void prepare_xreg_kernels();

void prepare_kernels() {
    prepare_w<float, 8>(); prepare_w<float, 16>(); prepare_w<float, 32>();
    prepare_w<double, 8>(); prepare_w<double, 16>(); prepare_w<double, 32>();
    allow_smem(k_slab_fwd_r<8, true, true>);
    allow_smem(k_slab_fwd_r<8, true, false>);
    allow_smem(k_slab_fwd_r<8, false, true>);
    allow_smem(k_slab_fwd_r<8, false, false>);
    allow_smem(k_slab_inv_r<8, true, true>);
    allow_smem(k_slab_inv_r<8, true, false>);
    allow_smem(k_slab_inv_r<8, false, true>);
    allow_smem(k_slab_inv_r<8, false, false>);
    allow_smem(k_slab_fwd_r<16, true, true>);
    allow_smem(k_slab_fwd_r<16, true, false>);
    allow_smem(k_slab_fwd_r<16, false, true>);
    allow_smem(k_slab_fwd_r<16, false, false>);
    allow_smem(k_slab_inv_r<16, true, true>);
    allow_smem(k_slab_inv_r<16, true, false>);
    allow_smem(k_slab_inv_r<16, false, true>);
    allow_smem(k_slab_inv_r<16, false, false>);
    prepare_far_kernels();
    prepare_xreg_kernels();
}

template bool launch_matvec<float>(const LatticeDev&, const MatvecArgs<float>&, cudaStream_t);
template bool launch_matvec<double>(const LatticeDev&, const MatvecArgs<double>&, cudaStream_t);

int matvec_passes(const LatticeDev& L, bool fp64) {
    return (fp64 ? pick_slab<double>(L) : pick_slab<float>(L)) ? 3 : 5;
}

size_t matvec_smem_bytes(const LatticeDev& L, bool fp64) {
    if (fp64) {
        const int wx = pick_xpass_w<double>(L);
        const int wz = pick_w([&](int w) { return smem_zpass<double>(L, w); });
        if (!wx || !wz) return 0;
        return smem_xpass<double>(L, wx);
    }
    const int wx = pick_xpass_w<float>(L);
    return wx ? smem_xpass<float>(L, wx) : 0;
}

void launch_dhat_build(const LatticeDev& L, int n_slot, const double2* kappa, double2* G, double2* Dr64, float2* Dr32,
                       cudaStream_t st, float2* Dx32) {
    const size_t M = (size_t)L.Mx * L.My * L.Mz;
    dim3 g1((unsigned)((M + 255) / 256), n_slot);
    count_launch();
    k_green<<<g1, 256, 0, st>>>(L, kappa, G);
    const int nb = n_slot * 6;
    axis_launch<double, false, 3>(G, nb, L.My, L.Mx, L.Mz, L.Mz, L.Mz, L.pz, L.tw64z, nullptr, 1, st);
    axis_launch<double, false, 1>(G, nb, L.My, L.Mx, L.Mz, L.My, L.My, L.py, L.tw64y, nullptr, 1, st);
    axis_launch<double, false, 2>(G, nb, L.My, L.Mx, L.Mz, L.Mx, L.Mx, L.px, L.tw64x, nullptr, 1, st);
    const size_t R = (size_t)L.Hx * L.Hy * L.Hz * 6 * n_slot;
    count_launch();
    k_extract<<<(unsigned)((R + 255) / 256), 256, 0, st>>>(L, n_slot, G, Dr64, Dr32);
    if (Dx32) launch_dhat_interleave(L, n_slot, Dr64, Dx32, st);
}

}  // namespace eels
