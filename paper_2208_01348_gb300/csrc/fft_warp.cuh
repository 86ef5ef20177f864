// Register-resident FFTs of 64 and 128 points, four lines per warp (FP32).
//
// Lane = q + 4p (q = 0..3 the line, p = 0..7) holds the elements p + 8r of
// its line in register r (r = 0..7 for 64 points, 0..15 for 128).  A length-8
// (64) or length-16 (128) DFT over the registers, the twiddles
// exp(-+2 pi i p k / L), a transpose among the 8 lanes of the line through a
// warp-private shared tile, and length-8 DFTs over the registers leave
// element j + 8m of the transform in register m of lane j: input and output
// use the same (lane, register) <-> index map, forward and inverse alike.
//
// HIN ("half input"): the registers r >= R/2 hold zeros (a lattice line that
// fills the first half of its zero-padded transform); the first radix-4 layer
// then runs on two inputs.  Twiddles come from a callable tw(k) returning
// exp(-2 pi i p k / L) for this lane (a shared table or registers).
#pragma once
#include "fft.cuh"

namespace eels {

constexpr int R64_QS = 132;   // transpose tile strides (8-byte units): line -> 4, lane -> 1 (mod 16)
constexpr int R64_PS = 17;
constexpr int R64_TILE = 4 * R64_QS;
constexpr int R128_QS = 148;  // transpose tile strides (8-byte units): line -> 4, lane -> 1 (mod 16)
constexpr int R128_PS = 17;
constexpr int R128_TILE = 4 * R128_QS;

// Length-4 DFT of (a, b, 0, 0): out = (a + b, a + rot(b), a - b, a - rot(b)),
// rot = multiplication by -i (forward) or +i (inverse).
template <bool INV>
__device__ __forceinline__ void dft4_half(float2 a, float2 b, float2 (&o)[4]) {
    const float2 rb = rot_mi<INV>(b);
    o[0] = a + b;
    o[1] = a + rb;
    o[2] = a - b;
    o[3] = a - rb;
}

// Length-8 DFT over v[0..7]; with HIN, v[4..7] are zero and not read.
template <bool INV, bool HIN>
__device__ __forceinline__ void dft8_reg(float2 (&v)[8]) {
    if constexpr (!HIN) {
        Dft<8, INV, float2>::run(v);
    } else {
        const float h = (float)K_SQRT_HALF;
        float2 e[4], o[4];
        dft4_half<INV>(v[0], v[2], e);
        dft4_half<INV>(v[1], v[3], o);
        float2 t1, t3;
        if (!INV) {
            t1.x = h * (o[1].x + o[1].y); t1.y = h * (o[1].y - o[1].x);
            t3.x = h * (o[3].y - o[3].x); t3.y = -h * (o[3].x + o[3].y);
        } else {
            t1.x = h * (o[1].x - o[1].y); t1.y = h * (o[1].y + o[1].x);
            t3.x = -h * (o[3].x + o[3].y); t3.y = h * (o[3].x - o[3].y);
        }
        const float2 t2 = rot_mi<INV>(o[2]);
        v[0] = e[0] + o[0]; v[4] = e[0] - o[0];
        v[1] = e[1] + t1;   v[5] = e[1] - t1;
        v[2] = e[2] + t2;   v[6] = e[2] - t2;
        v[3] = e[3] + t3;   v[7] = e[3] - t3;
    }
}

// Length-16 DFT over v[0..15] (n = n1 + 4 n2, k = k1 + 4 k2: length-4 DFTs
// over n2, twiddles w16^(n1 k1), length-4 DFTs over n1); with HIN,
// v[8..15] are zero and not read.
template <bool INV, bool HIN>
__device__ __forceinline__ void dft16_reg(float2 (&v)[16]) {
    float2 a[4][4];
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) {
        if constexpr (HIN) {
            dft4_half<INV>(v[n1], v[n1 + 4], a[n1]);
        } else {
            float2 t[4] = {v[n1], v[n1 + 4], v[n1 + 8], v[n1 + 12]};
            Dft<4, INV, float2>::run(t);
#pragma unroll
            for (int k1 = 0; k1 < 4; ++k1) a[n1][k1] = t[k1];
        }
    }
    // w16^(n1 k1) for n1 k1 in {1, 2, 3, 4, 6, 9}: cos/sin of multiples of pi/8
    const float c1 = 0.92387953251128675613f, s1 = 0.38268343236508977173f, h = 0.70710678118654752440f;
    const float sg = INV ? 1.f : -1.f;
    auto rot = [&](float2 x, float c, float s) { return make_float2(x.x * c - x.y * s * sg, x.x * s * sg + x.y * c); };
    a[1][1] = rot(a[1][1], c1, s1);        // w^1
    a[1][2] = rot(a[1][2], h, h);          // w^2
    a[1][3] = rot(a[1][3], s1, c1);        // w^3
    a[2][1] = rot(a[2][1], h, h);          // w^2
    a[2][2] = rot_mi<INV>(a[2][2]);        // w^4 = -+i
    a[2][3] = rot(a[2][3], -h, h);         // w^6
    a[3][1] = rot(a[3][1], s1, c1);        // w^3
    a[3][2] = rot(a[3][2], -h, h);         // w^6
    a[3][3] = rot(a[3][3], -c1, -s1);      // w^9
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        float2 t[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
        Dft<4, INV, float2>::run(t);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[k2];
    }
}

template <bool INV, bool HIN, class TW>
__device__ __forceinline__ void fft64_warp_t(float2 (&v)[8], float2* tile, int q, int p, TW tw) {
    dft8_reg<INV, HIN>(v);
#pragma unroll
    for (int k = 1; k < 8; ++k) {
        float2 w = tw(k);
        if (INV) w.y = -w.y;
        v[k] = v[k] * w;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) tile[q * R64_QS + p * R64_PS + k] = v[k];
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = tile[q * R64_QS + i * R64_PS + p];
    __syncwarp();
    Dft<8, INV, float2>::run(v);
}

template <bool INV, bool HIN, class TW>
__device__ __forceinline__ void fft128_warp_t(float2 (&v)[16], float2* tile, int q, int p, TW tw) {
    dft16_reg<INV, HIN>(v);
#pragma unroll
    for (int k = 1; k < 16; ++k) {
        float2 w = tw(k);
        if (INV) w.y = -w.y;
        v[k] = v[k] * w;
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) tile[q * R128_QS + p * R128_PS + k] = v[k];
    __syncwarp();
    float2 a[8], b[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        a[i] = tile[q * R128_QS + i * R128_PS + p];
        b[i] = tile[q * R128_QS + i * R128_PS + p + 8];
    }
    __syncwarp();
    Dft<8, INV, float2>::run(a);
    Dft<8, INV, float2>::run(b);
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) {
        v[2 * k2] = a[k2];
        v[2 * k2 + 1] = b[k2];
    }
}

// Twiddles from a shared table tw[t] = exp(-2 pi i t / L).
template <bool INV, bool HIN = false>
__device__ __forceinline__ void fft64_warp(float2 (&v)[8], float2* tile, int q, int p, const float2* tw) {
    fft64_warp_t<INV, HIN>(v, tile, q, p, [&](int k) { return tw[p * k]; });
}
template <bool INV, bool HIN = false>
__device__ __forceinline__ void fft128_warp(float2 (&v)[16], float2* tile, int q, int p, const float2* tw) {
    fft128_warp_t<INV, HIN>(v, tile, q, p, [&](int k) { return tw[p * k]; });
}

// One transform of L = 8 R points per line: the 64- or 128-point routine.
template <int R, bool INV, bool HIN, class TW>
__device__ __forceinline__ void fft_warp_t(float2 (&v)[R], float2* tile, int q, int p, TW tw) {
    if constexpr (R == 8) fft64_warp_t<INV, HIN>(v, tile, q, p, tw);
    else fft128_warp_t<INV, HIN>(v, tile, q, p, tw);
}

}  // namespace eels
