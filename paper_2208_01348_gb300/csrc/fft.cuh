// Shared-memory mixed-radix FFT core (radices 2, 3, 4, 5, 7, 8).
//
// Stockham auto-sort formulation (decimation in time, out of place between
// two shared-memory buffers): at a stage of radix R, with Ns the length of
// the sub-transforms already done, butterfly j (0 <= j < L/R) reads the R
// inputs a[j + r L/R], multiplies input r by w^(r k), k = j mod Ns,
// w = exp(-+2 pi i / (Ns R)), takes a length-R DFT and writes output r to
// b[(j / Ns) Ns R + k + r Ns].  After all stages the result is in natural
// order.  Forward uses exp(-2 pi i n k / L); the inverse is unnormalised.
//
// A batch of NL lines is transformed together: element i of line l lives at
// buf[l * lstride + i * estride], so the same routine serves lines stored
// contiguously (estride = 1) and lines interleaved across a tile
// (lstride = 1).  Twiddles come from a table tw[t] = exp(-2 pi i t / L).
#pragma once
#include "common.cuh"

namespace eels {

#define FFT_MAX_STAGES 12
#define FFT_MAX_LEN 512

// One Stockham stage: radix R after sub-transforms of length Ns; nb = L/R
// butterflies per line; ts = L/(Ns R) is the twiddle-table stride.  The
// shifts are log2 of Ns and nb when those are powers of two (else -1), so
// the index arithmetic of the common power-of-two lengths avoids divisions.
struct FftStage {
    int R, Ns, ns_shift, nb, nb_shift, ts;
};

struct FftPlan {
    int L;
    int nst;
    FftStage st[FFT_MAX_STAGES];
};

// sqrt(1/2), cos/sin(2 pi/3), and the R = 5, 7 roots of unity (values of
// elementary closed forms, e.g. cos(2 pi/5) = (sqrt 5 - 1)/4).
#define K_SQRT_HALF 0.70710678118654752440
#define K_C3 (-0.5)
#define K_S3 0.86602540378443864676
#define K_C5_1 0.30901699437494742410
#define K_S5_1 0.95105651629515357212
#define K_C5_2 (-0.80901699437494742410)
#define K_S5_2 0.58778525229247312917
#define K_C7_1 0.62348980185873353053
#define K_S7_1 0.78183148246802980871
#define K_C7_2 (-0.22252093395631440429)
#define K_S7_2 0.97492791218182360702
#define K_C7_3 (-0.90096886790241912624)
#define K_S7_3 0.43388373911755812048

// Length-R DFT in registers.  INV=false: X_p = sum_q v_q exp(-2 pi i p q / R).
template <int R, bool INV, typename C> struct Dft;

template <bool INV, typename C> struct Dft<2, INV, C> {
    __device__ __forceinline__ static void run(C* v) { C a = v[0], b = v[1]; v[0] = a + b; v[1] = a - b; }
};

template <bool INV, typename C> __device__ __forceinline__ C rot_mi(C a) { return INV ? mul_i(a) : mul_mi(a); }  // * exp(-+ i pi/2)

template <bool INV, typename C> struct Dft<4, INV, C> {
    __device__ __forceinline__ static void run(C* v) {
        C s0 = v[0] + v[2], d0 = v[0] - v[2];
        C s1 = v[1] + v[3], d1 = rot_mi<INV>(v[1] - v[3]);
        v[0] = s0 + s1; v[2] = s0 - s1;
        v[1] = d0 + d1; v[3] = d0 - d1;
    }
};

template <bool INV, typename C> struct Dft<8, INV, C> {
    __device__ __forceinline__ static void run(C* v) {
        using Rl = decltype(v[0].x);
        const Rl h = (Rl)K_SQRT_HALF;
        C e[4] = {v[0], v[2], v[4], v[6]};
        C o[4] = {v[1], v[3], v[5], v[7]};
        Dft<4, INV, C>::run(e);
        Dft<4, INV, C>::run(o);
        // twiddles exp(-+ 2 pi i p / 8), p = 1, 2, 3
        C t1, t3;
        if (!INV) {
            t1.x = h * (o[1].x + o[1].y); t1.y = h * (o[1].y - o[1].x);
            t3.x = h * (o[3].y - o[3].x); t3.y = -h * (o[3].x + o[3].y);
        } else {
            t1.x = h * (o[1].x - o[1].y); t1.y = h * (o[1].y + o[1].x);
            t3.x = -h * (o[3].x + o[3].y); t3.y = h * (o[3].x - o[3].y);
        }
        C t2 = rot_mi<INV>(o[2]);
        v[0] = e[0] + o[0]; v[4] = e[0] - o[0];
        v[1] = e[1] + t1;   v[5] = e[1] - t1;
        v[2] = e[2] + t2;   v[6] = e[2] - t2;
        v[3] = e[3] + t3;   v[7] = e[3] - t3;
    }
};

template <bool INV, typename C> struct Dft<3, INV, C> {
    __device__ __forceinline__ static void run(C* v) {
        using Rl = decltype(v[0].x);
        const Rl c = (Rl)K_C3, s = (Rl)(INV ? -K_S3 : K_S3);
        C a = v[1] + v[2], b = v[1] - v[2];
        C m = v[0] + c * a;
        C jb; jb.x = s * b.y; jb.y = -s * b.x;   // -i s b
        v[0] = v[0] + a;
        v[1] = m + jb;
        v[2] = m - jb;
    }
};

// Generic odd-length DFT (R = 5, 7) from symmetric pairs:
// X_p = v0 + sum_{q=1}^{(R-1)/2} [ (v_q + v_{R-q}) cos(2 pi p q/R) -+ i (v_q - v_{R-q}) sin(2 pi p q/R) ]
template <int R, bool INV, typename C> struct DftOdd {
    __device__ __forceinline__ static void run(C* v, const double* cs, const double* sn) {
        using Rl = decltype(v[0].x);
        constexpr int H = (R - 1) / 2;
        C sp[H], sm[H];
#pragma unroll
        for (int q = 1; q <= H; ++q) { sp[q - 1] = v[q] + v[R - q]; sm[q - 1] = v[q] - v[R - q]; }
        C out[R];
        C x0 = v[0];
#pragma unroll
        for (int q = 0; q < H; ++q) x0 = x0 + sp[q];
        out[0] = x0;
#pragma unroll
        for (int p = 1; p <= H; ++p) {
            C re = v[0], im; im.x = 0; im.y = 0;
#pragma unroll
            for (int q = 1; q <= H; ++q) {
                int m = (p * q) % R;
                Rl c = (Rl)cs[m], s = (Rl)sn[m];
                re = re + c * sp[q - 1];
                im = im + s * sm[q - 1];
            }
            // forward: -i * im ; inverse: +i * im
            C jim = INV ? mul_i(im) : mul_mi(im);
            out[p] = re + jim;
            out[R - p] = re - jim;
        }
#pragma unroll
        for (int p = 0; p < R; ++p) v[p] = out[p];
    }
};

template <bool INV, typename C> struct Dft<5, INV, C> {
    __device__ __forceinline__ static void run(C* v) {
        const double cs[5] = {1.0, K_C5_1, K_C5_2, K_C5_2, K_C5_1};
        const double sn[5] = {0.0, K_S5_1, K_S5_2, -K_S5_2, -K_S5_1};
        DftOdd<5, INV, C>::run(v, cs, sn);
    }
};
template <bool INV, typename C> struct Dft<7, INV, C> {
    __device__ __forceinline__ static void run(C* v) {
        const double cs[7] = {1.0, K_C7_1, K_C7_2, K_C7_3, K_C7_3, K_C7_2, K_C7_1};
        const double sn[7] = {0.0, K_S7_1, K_S7_2, K_S7_3, -K_S7_3, -K_S7_2, -K_S7_1};
        DftOdd<7, INV, C>::run(v, cs, sn);
    }
};

// One Stockham stage of radix R over NL lines.  LINE_FAST: adjacent
// threads take adjacent lines (good when lstride == 1).
template <int R, bool INV, bool LINE_FAST, int NL, typename C>
__device__ __forceinline__ void fft_stage(const C* __restrict__ a, C* __restrict__ b, int lstride, int estride,
                                          const FftStage sd, const C* __restrict__ tw) {
    const int nb = sd.nb, Ns = sd.Ns;
    const int total = NL * nb;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        int line, j;
        if (LINE_FAST) {
            line = t % NL;
            j = t / NL;
        } else if (sd.nb_shift >= 0) {
            j = t & (nb - 1);
            line = t >> sd.nb_shift;
        } else {
            j = t % nb;
            line = t / nb;
        }
        int k, jq;
        if (sd.ns_shift >= 0) {
            k = j & (Ns - 1);
            jq = j >> sd.ns_shift;
        } else {
            k = j % Ns;
            jq = j / Ns;
        }
        const C* src = a + line * lstride;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[(j + r * nb) * estride];
        if (Ns > 1) {
            const int step = k * sd.ts;
#pragma unroll
            for (int r = 1; r < R; ++r) {
                C w = tw[r * step];
                if (INV) w.y = -w.y;
                v[r] = v[r] * w;
            }
        }
        Dft<R, INV, C>::run(v);
        C* dst = b + line * lstride;
        const int base = jq * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[(base + r * Ns) * estride] = v[r];
    }
}

// Stage with arbitrary element access: inputs come from in(line, i), outputs
// go to out(line, i, value).  Used for the first and last stages, which read
// and write global memory (or another shared buffer) directly.
template <int R, bool INV, bool LINE_FAST, int NL, typename C, class In, class Out>
__device__ __forceinline__ void fft_stage_f(const FftStage sd, const C* __restrict__ tw, In in, Out out) {
    const int nb = sd.nb, Ns = sd.Ns;
    const int total = NL * nb;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        int line, j;
        if (LINE_FAST) {
            line = t % NL;
            j = t / NL;
        } else if (sd.nb_shift >= 0) {
            j = t & (nb - 1);
            line = t >> sd.nb_shift;
        } else {
            j = t % nb;
            line = t / nb;
        }
        int k, jq;
        if (sd.ns_shift >= 0) {
            k = j & (Ns - 1);
            jq = j >> sd.ns_shift;
        } else {
            k = j % Ns;
            jq = j / Ns;
        }
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = in(line, j + r * nb);
        if (Ns > 1) {
            const int step = k * sd.ts;
#pragma unroll
            for (int r = 1; r < R; ++r) {
                C w = tw[r * step];
                if (INV) w.y = -w.y;
                v[r] = v[r] * w;
            }
        }
        Dft<R, INV, C>::run(v);
        const int base = jq * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) out(line, base + r * Ns, v[r]);
    }
}

template <bool INV, bool LINE_FAST, int NL, typename C, class In, class Out>
__device__ __forceinline__ void fft_stage_any(const FftStage sd, const C* tw, In in, Out out) {
    switch (sd.R) {
        case 2: fft_stage_f<2, INV, LINE_FAST, NL>(sd, tw, in, out); break;
        case 3: fft_stage_f<3, INV, LINE_FAST, NL>(sd, tw, in, out); break;
        case 4: fft_stage_f<4, INV, LINE_FAST, NL>(sd, tw, in, out); break;
        case 5: fft_stage_f<5, INV, LINE_FAST, NL>(sd, tw, in, out); break;
        case 7: fft_stage_f<7, INV, LINE_FAST, NL>(sd, tw, in, out); break;
        default: fft_stage_f<8, INV, LINE_FAST, NL>(sd, tw, in, out); break;
    }
}

// Full transform of NL lines whose inputs are read through ld(line, i) by
// the first stage and whose outputs are handed to st(line, i, value) by the
// last stage; the stages in between ping-pong between the shared buffers A
// and B (element i of line l at l * lstride + i * estride; with PAD8 one
// padding slot follows every 8 elements, i -> i + i/8, which together with a
// line stride of 8 mod 16 makes the radix-8 stride-8 scatter of the first
// stage free of bank conflicts).  The block is synchronised between stages
// and after the last one.
template <bool INV, bool LINE_FAST, int NL, bool PAD8 = false, typename C, class Ld, class St>
__device__ void fft_lines_io(C* A, C* B, int lstride, int estride, const FftPlan& p, const C* tw, Ld ld, St st) {
    auto sm_in = [&](const C* buf) {
        return [=](int l, int i) { return buf[l * lstride + (PAD8 ? i + (i >> 3) : i) * estride]; };
    };
    auto sm_out = [&](C* buf) {
        return [=](int l, int i, C v) { buf[l * lstride + (PAD8 ? i + (i >> 3) : i) * estride] = v; };
    };
    if (p.nst == 1) {
        fft_stage_any<INV, LINE_FAST, NL>(p.st[0], tw, ld, st);
        __syncthreads();
        return;
    }
    fft_stage_any<INV, LINE_FAST, NL>(p.st[0], tw, ld, sm_out(A));
    __syncthreads();
    C* a = A;
    C* b = B;
    for (int s = 1; s + 1 < p.nst; ++s) {
        fft_stage_any<INV, LINE_FAST, NL>(p.st[s], tw, sm_in(a), sm_out(b));
        __syncthreads();
        C* t = a;
        a = b;
        b = t;
    }
    fft_stage_any<INV, LINE_FAST, NL>(p.st[p.nst - 1], tw, sm_in(a), st);
    __syncthreads();
}

// Full transform of NL lines; returns the buffer that holds the result (a
// or b).  Synchronises the block after every stage (callers sync before).
template <bool INV, bool LINE_FAST, int NL, typename C>
__device__ C* fft_lines(C* a, C* b, int lstride, int estride, const FftPlan& p, const C* tw) {
    for (int st = 0; st < p.nst; ++st) {
        const FftStage sd = p.st[st];
        switch (sd.R) {
            case 2: fft_stage<2, INV, LINE_FAST, NL>(a, b, lstride, estride, sd, tw); break;
            case 3: fft_stage<3, INV, LINE_FAST, NL>(a, b, lstride, estride, sd, tw); break;
            case 4: fft_stage<4, INV, LINE_FAST, NL>(a, b, lstride, estride, sd, tw); break;
            case 5: fft_stage<5, INV, LINE_FAST, NL>(a, b, lstride, estride, sd, tw); break;
            case 7: fft_stage<7, INV, LINE_FAST, NL>(a, b, lstride, estride, sd, tw); break;
            default: fft_stage<8, INV, LINE_FAST, NL>(a, b, lstride, estride, sd, tw); break;
        }
        __syncthreads();
        C* t = a;
        a = b;
        b = t;
    }
    return a;
}

}  // namespace eels
