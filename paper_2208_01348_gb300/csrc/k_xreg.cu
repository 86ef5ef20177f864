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
#include <cuda.h>

#include <mutex>

#include "fft_warp.cuh"
#include "kernels.h"

namespace eels {

// Bulk copies and their mbarrier (sm_90+ PTX).  Every wait is bounded: a
// wait that gives up counts into g_wait_timeouts, which the host reads
// after a solve (EELS_E_TIMEOUT).
__device__ unsigned int g_wait_timeouts = 0;

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// The calling thread announces `bytes` of transfer on the barrier.
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// 1-D bulk copy global -> shared, completing on the barrier (16-byte aligned
// addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// 4-D tiled tensor copies (TMA) described by a tensor map in kernel-parameter
// space: global -> shared completing on the barrier, and shared -> global in
// the calling thread's bulk async-group.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_store_4d(const CUtensorMap* map, int c0, int c1, int c2, int c3, const void* src) {
    asm volatile(
        "cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4}], [%5];" ::"l"(
            reinterpret_cast<unsigned long long>(map)),
        "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(src))
        : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Wait until at most N of this thread's bulk groups still read shared memory.
template <int N> __device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
// Writes of this thread to shared memory become visible to the async proxy
// (a following bulk store reads them).
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Waits for phase `parity` of the barrier, at most `limit` polls.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, unsigned limit) {
    const unsigned addr = smem_u32(bar);
    for (unsigned i = 0; i < limit; ++i) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

constexpr int XR_WARPS = 4;
constexpr int XR_THREADS = 32 * XR_WARPS;
constexpr unsigned XR_WAIT_POLLS = 1u << 22;

template <int MX> struct XReg {
    static constexpr bool SPLIT = MX == 128;
    static constexpr int LPW = SPLIT ? 2 : 4;           // kz columns per warp
    static constexpr int ZT = LPW * XR_WARPS;           // kz' rows of D-hat per block
    static constexpr int HX = MX / 2 + 1;
    // shared row stride of the D-hat tile (8-byte words): the lanes of a load
    // differ in row by (lane & 1) (Mx = 128) or (lane & 3) (Mx = 64) and in
    // kx' by 2p + h or p, so a stride of 8 or 4 mod 16 puts the 16 lanes of
    // each half-warp on distinct bank pairs
    static constexpr int RS = SPLIT ? ((6 * HX + 7) / 16 * 16 + 8) : ((6 * HX + 11) / 16 * 16 + 4);
};
static_assert(XReg<128>::RS % 16 == 8 && XReg<128>::RS >= 6 * XReg<128>::HX, "row stride");
static_assert(XReg<64>::RS % 16 == 4 && XReg<64>::RS >= 6 * XReg<64>::HX, "row stride");

// One block per D-hat octant tile (ky' = blockIdx.y, kz' in [z0, z0 + ZT))
// and group of systems (a.spb consecutive systems, blockIdx.z).  The tile
// (and, in the first tile, the row kz' = Mz/2) comes into shared memory by
// bulk copies and serves every (ky, kz) whose octant image lies in it: ky in
// {ky', My - ky'} and kz in {kz', Mz - kz'} -- up to four passes over ZT kz
// columns; the column kz' = 0, its own mirror, hands its mirror pass to
// kz = Mz/2.  The systems of the group that share the tile's energy (the
// beams of one energy) reuse it: it is copied again only when the system's
// D-hat slot changes.  The last tile may be partial (Mz/2 not a multiple of
// ZT): its columns past Mz/2 idle.
template <int MX>
__global__ void __launch_bounds__(XR_THREADS, 4) k_xpass_reg(LatticeDev L, MatvecArgs<float> a) {
    using X = XReg<MX>;
    constexpr bool SPLIT = X::SPLIT;
    constexpr int ZT = X::ZT;
    __shared__ float2 tws[MX];                          // exp(-2 pi i t / MX)
    __shared__ float2 tw2[7 * 8];                       // w64^(p k) at [k - 1][p]: lanes p read consecutive words
    __shared__ float2 tiles[XR_WARPS][R64_TILE];
    __shared__ __align__(16) float2 dt[(ZT + 1) * X::RS];
    __shared__ __align__(8) unsigned long long bar;
    const int kyr = blockIdx.y, z0 = blockIdx.x * ZT;
    const int Mz = L.Mz, Nx = L.Nx, My = L.My, Hx = L.Hx;
    const int s_begin = blockIdx.z * a.spb, s_end = min(a.S, s_begin + a.spb);
    const size_t row = (size_t)6 * Hx;                  // float2 per kz' row of D-hat (= 6 HX)
    const int nrow = min(ZT, Mz / 2 - z0);              // rows of this tile
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    for (int t = threadIdx.x; t < MX; t += XR_THREADS) tws[t] = L.tw32x[t];
    for (int t = threadIdx.x; t < 7 * 8; t += XR_THREADS) tw2[t] = L.tw32x[(MX / 64) * (t & 7) * ((t >> 3) + 1)];
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, q = lane & 3, p = lane >> 2;
    const int h = SPLIT ? (q >> 1) : 0;                 // frequency parity (Mx = 128)
    const int j = warp * X::LPW + (SPLIT ? (q & 1) : q);   // this lane's column of the tile
    float2* tile = tiles[warp];
    auto tw = [&](int k) { return tw2[(k - 1) * 8 + p]; };   // w64^(p k)
    const size_t plane = (size_t)Nx * Mz;
    const size_t cstride = (size_t)My * plane;
    const float2 zero = make_float2(0.f, 0.f);
    constexpr int RIN = SPLIT ? 8 : 4;                  // registers that can hold lattice rows
    const int nky = (kyr == 0 || 2 * kyr == My) ? 1 : 2;
    int cur_slot = -1;
    unsigned phase = 0;

    for (int s = s_begin; s < s_end; ++s) {
        if (a.active && !a.active[s]) continue;
        const int slot = a.sys_slot[s];
        if (slot != cur_slot) {
            // (re)fill the tile: every thread is done reading the previous one
            __syncthreads();
            if (threadIdx.x == 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                // one bulk copy per row (rows are 48 Hx bytes: 16-byte
                // multiples) into rows of RS words
                const float2* src = a.Dx + (((size_t)slot * L.Hy + kyr) * L.Hz + z0) * row;
                const unsigned rb = (unsigned)(row * sizeof(float2));
                mbar_expect_tx(&bar, rb * (nrow + (z0 == 0 ? 1 : 0)));
                for (int r = 0; r < nrow; ++r) bulk_g2s(dt + r * X::RS, src + r * row, rb, &bar);
                if (z0 == 0) bulk_g2s(dt + ZT * X::RS, src + (size_t)(Mz / 2) * row, rb, &bar);
            }
            // the block decides together, so that no warp leaves while others wait at a barrier
            if (__syncthreads_or(!mbar_wait(&bar, phase, XR_WAIT_POLLS))) {
                // give up: record it, let the copies land before the block's
                // shared memory is released, and leave
                if (threadIdx.x == 0) {
                    atomicAdd(&g_wait_timeouts, 1u);
                    mbar_wait(&bar, phase, XR_WAIT_POLLS);
                }
                return;
            }
            phase ^= 1u;
            cur_slot = slot;
        }
        for (int pass = 0; pass < 2 * nky; ++pass) {
            const int ky = (pass >> 1) ? My - kyr : kyr;
            const bool mirror = pass & 1;
            const bool nyq = mirror && z0 + j == 0;      // kz' = 0 hands its mirror pass to kz = Mz/2
            const bool col_ok = z0 + j < Mz / 2;         // a column of a partial tile may idle
            const int kz = !mirror ? z0 + j : (nyq ? Mz / 2 : Mz - (z0 + j));
            const int drow = nyq ? ZT : j;
            const float sy = (pass >> 1) ? -1.f : 1.f;
            const float sz = (mirror && !nyq) ? -1.f : 1.f, syz = sy * sz;

            float2* U0 = a.U + ((size_t)s * 3 * My + ky) * plane + (col_ok ? kz : 0);
            float2 v[3][8];
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const int ix = p + 8 * r;
                    v[c][r] = (r < RIN && ix < Nx && col_ok) ? U0[c * cstride + (size_t)ix * Mz] : zero;
                }
            if constexpr (SPLIT) {                      // odd frequencies: x_n w128^n
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const float2 w = h ? tws[p + 8 * r] : make_float2(1.f, 0.f);
#pragma unroll
                    for (int c = 0; c < 3; ++c) v[c][r] = v[c][r] * w;
                }
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) fft64_warp_t<false, !SPLIT>(v[c], tile, q, p, tw);

            // D-hat product at kx = p + 8m (Mx = 64) or 2 (p + 8m) + h (Mx = 128):
            // octant index kx', and the sign sx of the odd components (-1 for
            // m >= 4, where kx >= MX/2; at kx = MX/2 those components vanish)
            const float2* Dk = dt + (col_ok ? drow : 0) * X::RS;
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const int kx = SPLIT ? 2 * (p + 8 * m) + h : p + 8 * m;
                const int kxr = m < 4 ? kx : MX - kx;
                const float sx = m < 4 ? 1.f : -1.f;
                const float2* d = Dk + kxr;
                const float2 dxx = d[0];
                const float2 dxy = (sx * sy) * d[Hx];
                const float2 dxz = (sx * sz) * d[2 * Hx];
                const float2 dyy = d[3 * Hx];
                const float2 dyz = syz * d[4 * Hx];
                const float2 dzz = d[5 * Hx];
                const float2 Xv = v[0][m], Yv = v[1][m], Zv = v[2][m];
                v[0][m] = dxx * Xv + dxy * Yv + dxz * Zv;
                v[1][m] = dxy * Xv + dyy * Yv + dyz * Zv;
                v[2][m] = dxz * Xv + dyz * Yv + dzz * Zv;
            }

#pragma unroll
            for (int c = 0; c < 3; ++c) fft64_warp_t<true, false>(v[c], tile, q, p, tw);
            if constexpr (SPLIT) {
                // y_n = z0_n + w128^(-n) z1_n: the h = 1 lane twiddles its z1,
                // lane h = 0 stores rows r < 4 and lane h = 1 rows r >= 4, each
                // receiving the partner's half with one shuffle
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
                    for (int jj = 0; jj < 4; ++jj) {
                        const float2 send = h ? v[c][jj] : v[c][jj + 4];
                        const float2 mine = h ? v[c][jj + 4] : v[c][jj];
                        float2 got;
                        got.x = __shfl_xor_sync(0xffffffffu, send.x, 2);
                        got.y = __shfl_xor_sync(0xffffffffu, send.y, 2);
                        const int ix = p + 8 * (jj + 4 * h);
                        if (ix < Nx && col_ok) U0[c * cstride + (size_t)ix * Mz] = mine + got;
                    }
            } else {
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const int ix = p + 8 * r;
                        if (ix < Nx && col_ok) U0[c * cstride + (size_t)ix * Mz] = v[c][r];
                    }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// The same x pass with the U lines moved by the tensor memory accelerator.
//
// When Mz is a multiple of 2 ZT, the kz lines pair into aligned tiles: the
// direct tile kz in [z0, z0 + ZT) (kz' = kz) and the mirror tile
// kz in [Mz - z0 - ZT, Mz - z0) (kz' = Mz - kz in (z0, z0 + ZT]); both use
// the D-hat rows kz' in [z0, z0 + ZT], and every kz (kz = Mz/2 included, in
// the mirror tile of the last z0) belongs to exactly one tile.  A pass moves
// the three components of one tile, Nx rows x ZT kz each, into shared memory
// with one 4-D tensor copy (box ZT x Nx x 1 x 3 of U viewed as
// [3S][My][Nx][Mz]), transforms it in registers as k_xpass_reg does, writes
// the results back into the same buffer (each warp owns its columns) and
// stores the tile with one tensor copy; two buffers let the copy of the next
// pass overlap the current one.
// ---------------------------------------------------------------------------
template <int MX> struct XTma {
    static constexpr int ZT = XReg<MX>::ZT;
    static constexpr int TILE = 3 * (MX / 2) * ZT;      // float2 of a U tile (Nx <= MX/2)
    // The tensor copies swizzle the tile's rows so that the rows p + 8r and
    // columns of a warp's access fall on distinct banks: Mx = 128, rows of
    // ZT = 8 elements (64 bytes), the 64-byte swizzle (the 16-byte chunk index
    // within a row XORed with bits 1-2 of the row index); Mx = 64, rows of
    // ZT = 16 elements (128 bytes), the 128-byte swizzle (XORed with bits 0-2)
    static constexpr int ROW_SHIFT = MX == 128 ? 1 : 0;
    static constexpr int CHUNKS = MX == 128 ? 4 : 8;     // 16-byte chunks per row
};

// Dynamic shared memory of k_xpass_tma (above the 48 KB of static arrays).
template <int MX> struct XTmaSmem {
    float2 ut[2][XTma<MX>::TILE];                       // U tiles (tensor-copy destinations, 1024-byte aligned)
    float2 dt[(XReg<MX>::ZT + 1) * XReg<MX>::RS];      // D-hat rows kz' in [z0, z0 + ZT]
    float2 tiles[XR_WARPS][R64_TILE];                   // warp-private transposes
    float2 tws[MX];
    float2 tw2[7 * 8];
    unsigned long long bar_d, bar_u[2];
};

struct XPass {
    int s, ky, mirror;
};

template <int MX>
__global__ void __launch_bounds__(XR_THREADS, 3)
k_xpass_tma(LatticeDev L, MatvecArgs<float> a, const __grid_constant__ CUtensorMap umap) {
    using X = XReg<MX>;
    constexpr bool SPLIT = X::SPLIT;
    constexpr int ZT = X::ZT;
    extern __shared__ __align__(1024) unsigned char xt_smem[];
    // the swizzled tensor copies want 1024-byte aligned buffers: align the
    // block's window explicitly (one spare KB is allocated for it)
    const unsigned pad = (1024u - (smem_u32(xt_smem) & 1023u)) & 1023u;
    XTmaSmem<MX>& sm = *reinterpret_cast<XTmaSmem<MX>*>(xt_smem + pad);
    auto& ut = sm.ut;
    auto& dt = sm.dt;
    auto& tiles = sm.tiles;
    auto& tws = sm.tws;
    auto& tw2 = sm.tw2;
    auto& bar_d = sm.bar_d;
    auto& bar_u = sm.bar_u;
    const int kyr = blockIdx.y, z0 = blockIdx.x * ZT;
    const int Mz = L.Mz, Nx = L.Nx, My = L.My, Hx = L.Hx;
    const int s_begin = blockIdx.z * a.spb, s_end = min(a.S, s_begin + a.spb);
    const size_t row = (size_t)6 * Hx;
    const int nky = (kyr == 0 || 2 * kyr == My) ? 1 : 2;
    const int per_sys = 2 * nky;                        // passes per system: ky choices x {direct, mirror}
    const unsigned tile_bytes = (unsigned)(3 * Nx * ZT * sizeof(float2));
    // pass i of the block: its system (skipping inactive ones), ky and tile
    auto pass_of = [&](int i, XPass& ps) -> bool {
        int s = s_begin, k = i;
        for (; s < s_end; ++s) {
            if (a.active && !a.active[s]) continue;
            if (k < per_sys) break;
            k -= per_sys;
        }
        if (s >= s_end) return false;
        ps.s = s;
        ps.ky = (k >> 1) ? My - kyr : kyr;
        ps.mirror = k & 1;
        return true;
    };
    auto issue_load = [&](const XPass& ps, int b) {
        const int kz0 = ps.mirror ? Mz - z0 - ZT : z0;
        mbar_expect_tx(&bar_u[b], tile_bytes);
        tma_load_4d(ut[b], &umap, kz0, 0, ps.ky, 3 * ps.s, &bar_u[b]);
    };
    XPass cur{};
    const bool any = pass_of(0, cur);
    if (threadIdx.x == 0) {
        mbar_init(&bar_d, 1);
        mbar_init(&bar_u[0], 1);
        mbar_init(&bar_u[1], 1);
        if (any) issue_load(cur, 0);
    }
    for (int t = threadIdx.x; t < MX; t += XR_THREADS) tws[t] = L.tw32x[t];
    for (int t = threadIdx.x; t < 7 * 8; t += XR_THREADS) tw2[t] = L.tw32x[(MX / 64) * (t & 7) * ((t >> 3) + 1)];
    __syncthreads();
    if (!any) return;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, q = lane & 3, p = lane >> 2;
    const int h = SPLIT ? (q >> 1) : 0;
    const int j = warp * X::LPW + (SPLIT ? (q & 1) : q);   // this lane's column of the tile
    float2* tile = tiles[warp];
    auto tw = [&](int k) { return tw2[(k - 1) * 8 + p]; };
    const float2 zero = make_float2(0.f, 0.f);
    constexpr int RIN = SPLIT ? 8 : 4;
    // element of (component c, row ix, this lane's column j) in a U tile
    auto uidx = [&](int c, int ix) -> int {
        const int r = c * Nx + ix;
        constexpr int sh = XTma<MX>::ROW_SHIFT, mk = XTma<MX>::CHUNKS - 1;
        return r * ZT + ((((j >> 1) ^ ((r >> sh) & mk)) << 1) | (j & 1));
    };
    int cur_slot = -1;
    unsigned ph_d = 0, ph_u[2] = {0, 0};
    bool failed = false;

    for (int i = 0;; ++i) {
        const int b = i & 1;
        // the D-hat tile of this pass's energy
        const int slot = a.sys_slot[cur.s];
        if (slot != cur_slot) {
            __syncthreads();                             // every thread is done with the previous tile
            if (threadIdx.x == 0) {
                fence_async_shared();
                const float2* src = a.Dx + (((size_t)slot * L.Hy + kyr) * L.Hz + z0) * row;
                const unsigned rb = (unsigned)(row * sizeof(float2));
                mbar_expect_tx(&bar_d, rb * (ZT + 1));
                for (int r = 0; r <= ZT; ++r) bulk_g2s(dt + r * X::RS, src + r * row, rb, &bar_d);
            }
            // the block decides together, so that no warp leaves while others wait at a barrier
            if (__syncthreads_or(!mbar_wait(&bar_d, ph_d, XR_WAIT_POLLS))) { failed = true; break; }
            ph_d ^= 1u;
            cur_slot = slot;
        }
        // prefetch the next pass's tile into the other buffer, once the store
        // that last read that buffer is done with it
        XPass nxt{};
        const bool more = pass_of(i + 1, nxt);
        if (threadIdx.x == 0 && more) {
            bulk_wait_read<0>();
            issue_load(nxt, b ^ 1);
        }
        if (__syncthreads_or(!mbar_wait(&bar_u[b], ph_u[b], XR_WAIT_POLLS))) { failed = true; break; }
        ph_u[b] ^= 1u;

        const bool mirror = cur.mirror;
        const int drow = mirror ? ZT - j : j;           // kz' - z0
        const bool nyq = mirror && z0 + ZT == Mz / 2 && j == 0;   // kz = Mz/2
        const float sy = cur.ky == kyr ? 1.f : -1.f;
        const float sz = (mirror && !nyq) ? -1.f : 1.f, syz = sy * sz;
        float2* T = ut[b];
        float2 v[3][8];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const int ix = p + 8 * r;
                v[c][r] = (r < RIN && ix < Nx) ? T[uidx(c, ix)] : zero;
            }
        if constexpr (SPLIT) {
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const float2 w = h ? tws[p + 8 * r] : make_float2(1.f, 0.f);
#pragma unroll
                for (int c = 0; c < 3; ++c) v[c][r] = v[c][r] * w;
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) fft64_warp_t<false, !SPLIT>(v[c], tile, q, p, tw);
        const float2* Dk = dt + drow * X::RS;
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int kx = SPLIT ? 2 * (p + 8 * m) + h : p + 8 * m;
            const int kxr = m < 4 ? kx : MX - kx;
            const float sx = m < 4 ? 1.f : -1.f;
            const float2* d = Dk + kxr;
            const float2 dxx = d[0];
            const float2 dxy = (sx * sy) * d[Hx];
            const float2 dxz = (sx * sz) * d[2 * Hx];
            const float2 dyy = d[3 * Hx];
            const float2 dyz = syz * d[4 * Hx];
            const float2 dzz = d[5 * Hx];
            const float2 Xv = v[0][m], Yv = v[1][m], Zv = v[2][m];
            v[0][m] = dxx * Xv + dxy * Yv + dxz * Zv;
            v[1][m] = dxy * Xv + dyy * Yv + dyz * Zv;
            v[2][m] = dxz * Xv + dyz * Yv + dzz * Zv;
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) fft64_warp_t<true, false>(v[c], tile, q, p, tw);
        // results into this warp's columns of the buffer (rows past Nx untouched)
        if constexpr (SPLIT) {
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
                for (int jj = 0; jj < 4; ++jj) {
                    const float2 send = h ? v[c][jj] : v[c][jj + 4];
                    const float2 mine = h ? v[c][jj + 4] : v[c][jj];
                    float2 got;
                    got.x = __shfl_xor_sync(0xffffffffu, send.x, 2);
                    got.y = __shfl_xor_sync(0xffffffffu, send.y, 2);
                    const int ix = p + 8 * (jj + 4 * h);
                    if (ix < Nx) T[uidx(c, ix)] = mine + got;
                }
        } else {
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int ix = p + 8 * r;
                    if (ix < Nx) T[uidx(c, ix)] = v[c][r];
                }
        }
        fence_async_shared();
        __syncthreads();
        if (threadIdx.x == 0) {
            tma_store_4d(&umap, mirror ? Mz - z0 - ZT : z0, 0, cur.ky, 3 * cur.s, T);
            bulk_commit();
        }
        if (!more) break;
        cur = nxt;
    }
    if (threadIdx.x == 0) {
        if (failed) atomicAdd(&g_wait_timeouts, 1u);
        // copies in flight must land before the block's shared memory is released
        bulk_wait_read<0>();
        if (failed) {
            mbar_wait(&bar_d, ph_d, XR_WAIT_POLLS);
            mbar_wait(&bar_u[0], ph_u[0], XR_WAIT_POLLS);
            mbar_wait(&bar_u[1], ph_u[1], XR_WAIT_POLLS);
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
    return (L.Mx == 64 || L.Mx == 128) && 2 * L.Nx <= L.Mx && L.Mz % 2 == 0;
}

namespace {

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled through the runtime's driver entry point (nullptr
// when the driver does not offer it: the x pass then loads U directly).
EncodeTiled encode_tiled() {
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(f);
        cudaGetLastError();
    });
    return fn;
}

// U viewed as [3S][My][Nx][Mz] of 8-byte elements, box ZT x Nx x 1 x 3
// (the 64-byte swizzle for 64-byte box rows, the 128-byte swizzle for
// 128-byte rows, as the tile indexing of k_xpass_tma expects).
bool u_tensor_map(const LatticeDev& L, const MatvecArgs<float>& a, int zt, CUtensorMap* map) {
    EncodeTiled enc = encode_tiled();
    if (!enc) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)L.Mz, (cuuint64_t)L.Nx, (cuuint64_t)L.My, (cuuint64_t)3 * a.S};
    const cuuint64_t strides[3] = {(cuuint64_t)L.Mz * 8, (cuuint64_t)L.Nx * L.Mz * 8,
                                   (cuuint64_t)L.My * L.Nx * L.Mz * 8};
    const cuuint32_t box[4] = {(cuuint32_t)zt, (cuuint32_t)L.Nx, 1, 3};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, (void*)a.U, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, zt == 8 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int MX>
bool launch_tma(const LatticeDev& L, const MatvecArgs<float>& a, int spb, unsigned groups, cudaStream_t st) {
    constexpr int ZT = XReg<MX>::ZT;
    if (L.Mz % (2 * ZT) != 0 || ((uintptr_t)a.U & 15) != 0) return false;
    CUtensorMap map;
    if (!u_tensor_map(L, a, ZT, &map)) return false;
    MatvecArgs<float> b = a;
    b.spb = spb;
    count_launch();
    k_xpass_tma<MX><<<dim3(L.Mz / 2 / ZT, L.Hy, groups), XR_THREADS, sizeof(XTmaSmem<MX>) + 1024, st>>>(L, b, map);
    return true;
}

}  // namespace

void prepare_xreg_kernels() {
    cudaFuncSetAttribute(k_xpass_tma<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(XTmaSmem<64>) + 1024);
    cudaFuncSetAttribute(k_xpass_tma<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(XTmaSmem<128>) + 1024);
}

bool launch_xpass_reg(const LatticeDev& L, const MatvecArgs<float>& a, cudaStream_t st) {
    if (!a.Dx || !xpass_reg_supported(L)) return false;
    const int spb = a.spb > 0 ? a.spb : 1;
    const unsigned groups = (unsigned)((a.S + spb - 1) / spb);
    if (L.xmode != 1 && (L.Mx == 64 ? launch_tma<64>(L, a, spb, groups, st) : launch_tma<128>(L, a, spb, groups, st)))
        return true;
    MatvecArgs<float> b = a;
    b.spb = spb;
    count_launch();
    if (L.Mx == 64) {
        constexpr int ZT = XReg<64>::ZT;
        k_xpass_reg<64><<<dim3((L.Mz / 2 + ZT - 1) / ZT, L.Hy, groups), XR_THREADS, 0, st>>>(L, b);
    } else {
        constexpr int ZT = XReg<128>::ZT;
        k_xpass_reg<128><<<dim3((L.Mz / 2 + ZT - 1) / ZT, L.Hy, groups), XR_THREADS, 0, st>>>(L, b);
    }
    return true;
}

void autotune_xreg(const LatticeDev& L, const MatvecArgs<float>& a, int max_spb, cudaStream_t st, int* mode, int* spb,
                   std::vector<std::array<float, 3>>* log) {
    *mode = 0;
    *spb = 1;
    if (log) log->clear();
    if (!a.Dx || !xpass_reg_supported(L)) return;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return; }
    float best = -1.f;
    for (int m : {1, 2}) {
        for (int b : {1, 2, 4, 8, 16}) {
            if (b > 1 && b > max_spb) break;
            LatticeDev Lc = L;
            Lc.xmode = m;
            MatvecArgs<float> ac = a;
            ac.spb = b;
            if (m == 2) {                                // tensor copies only where they apply
                CUtensorMap map;
                constexpr int zt64 = XReg<64>::ZT, zt128 = XReg<128>::ZT;
                const int zt = L.Mx == 64 ? zt64 : zt128;
                if (L.Mz % (2 * zt) != 0 || !u_tensor_map(L, a, zt, &map)) break;
            }
            launch_xpass_reg(Lc, ac, st);                // warm-up
            cudaEventRecord(e0, st);
            for (int r = 0; r < 3; ++r) launch_xpass_reg(Lc, ac, st);
            cudaEventRecord(e1, st);
            float ms = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            if (log) log->push_back({(float)m, (float)b, ms});
            if (best < 0.f || ms < best) { best = ms; *mode = m; *spb = b; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
}

unsigned int wait_timeouts() {
    unsigned int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_wait_timeouts, sizeof(v)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return v;
}

void launch_dhat_interleave(const LatticeDev& L, int n_slot, const double2* Dr64, float2* Dx, cudaStream_t st) {
    const size_t n = (size_t)L.Hx * L.Hy * L.Hz * 6 * n_slot;
    count_launch();
    k_dhat_interleave<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(L, n_slot, Dr64, Dx);
}

}  // namespace eels
