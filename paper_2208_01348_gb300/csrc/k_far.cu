// CL far field (Eq. 42 of the paper): for every direction n of the
// quadrature grid,
//   F'(n) = (I - n n) sum_j u_j exp(-i kappa n . r'_j)
// with r' in units of d and kappa = k d, and the reduction
//   sum_n w_n |F'(n)|^2.
// One thread per direction.  The lattice phase factorises,
// exp(-i kappa n.r') = exp(-i kappa (n_x x' + n_y y')) exp(-i kappa n_z z'),
// so each thread evaluates one exponential per (direction, column) and walks
// the column with a constant step factor exp(-i kappa n_z).  Column dipoles
// are staged in shared memory and read by every thread (broadcast).
// The columns of one staged round are summed in the working precision and
// each round's sum is added in FP64 (this part's FP64 rate is a small
// fraction of its FP32 rate: FP64 work per column would bound the kernel).
#include "solve.h"

namespace eels {

template <typename Rl> __device__ __forceinline__ cx<Rl> expmi(double2 kap, Rl phi);
// exp(-i kappa phi) = exp(Im(kappa) phi) (cos(Re kappa phi) - i sin(Re kappa phi))
template <> __device__ __forceinline__ float2 expmi<float>(double2 kap, float phi) {
    float s, c;
    sincosf((float)kap.x * phi, &s, &c);
    const float m = expf((float)kap.y * phi);
    return make_float2(m * c, -m * s);
}
template <> __device__ __forceinline__ double2 expmi<double>(double2 kap, double phi) {
    double s, c;
    sincos(kap.x * phi, &s, &c);
    const double m = exp(kap.y * phi);
    return make_double2(m * c, -m * s);
}

constexpr int FAR_THREADS = 128;
constexpr int FAR_CC = 8;   // columns staged per round

template <typename Rl>
__global__ void __launch_bounds__(FAR_THREADS) k_far(LatticeDev L, const cx<Rl>* u, const double2* kappa_sys,
                                                     const double* dirs, const double* wts, int n_dir, double* part) {
    using C = cx<Rl>;
    const int s = blockIdx.y;
    const int dn = blockIdx.x * FAR_THREADS + threadIdx.x;
    const bool valid = dn < n_dir;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* col = reinterpret_cast<C*>(smem_raw);   // [FAR_CC][3][Nz]
    const int Nz = L.Nz;
    const double2 kap = kappa_sys[s];
    double n[3] = {0, 0, 0};
    double w = 0;
    if (valid) { n[0] = dirs[3 * dn]; n[1] = dirs[3 * dn + 1]; n[2] = dirs[3 * dn + 2]; w = wts[dn]; }
    const C step = cvt<C>(expmi<double>(kap, n[2]));
    const Rl nx = (Rl)n[0], ny = (Rl)n[1], nz = (Rl)n[2];
    double2 S[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
    const size_t N = (size_t)L.N;
    const C* us = u + (size_t)s * 3 * N;
    const int ncol = L.Nx * L.Ny;
    for (int c0 = 0; c0 < ncol; c0 += FAR_CC) {
        __syncthreads();
        for (int t = threadIdx.x; t < FAR_CC * 3 * Nz; t += blockDim.x) {
            const int iz = t % Nz, c = (t / Nz) % 3, cc = t / (3 * Nz), colid = c0 + cc;
            C v = mk<C>(0.0, 0.0);
            if (colid < ncol) {
                const int dip = L.cellmap[((size_t)(colid % L.Nx) * L.Ny + colid / L.Nx) * L.Nz + iz];
                if (dip >= 0) v = us[(size_t)c * N + dip];
            }
            col[(cc * 3 + c) * Nz + iz] = v;
        }
        __syncthreads();
        if (!valid) continue;
        C R0 = mk<C>(0.0, 0.0), R1 = R0, R2 = R0;     // this round's columns
        for (int cc = 0; cc < FAR_CC; ++cc) {
            const int colid = c0 + cc;
            if (colid >= ncol) break;
            const int2 rg = L.col_range[colid];
            if (rg.x >= rg.y) continue;
            const int ix = colid % L.Nx, iy = colid / L.Nx;
            // cell centres relative to the lattice centre (exact in either precision)
            const Rl xr = (Rl)(2 * ix + 1 - L.Nx) * (Rl)0.5, yr = (Rl)(2 * iy + 1 - L.Ny) * (Rl)0.5,
                     zr = (Rl)(2 * rg.x + 1 - Nz) * (Rl)0.5;
            C e = expmi<Rl>(kap, nx * xr + ny * yr + nz * zr);
            C T0 = mk<C>(0.0, 0.0), T1 = T0, T2 = T0;
            const C* cx0 = col + (cc * 3) * Nz;
            for (int iz = rg.x; iz < rg.y; ++iz) {
                T0 = T0 + e * cx0[iz];
                T1 = T1 + e * cx0[Nz + iz];
                T2 = T2 + e * cx0[2 * Nz + iz];
                e = e * step;
            }
            R0 = R0 + T0;
            R1 = R1 + T1;
            R2 = R2 + T2;
        }
        S[0] = S[0] + widen(R0);
        S[1] = S[1] + widen(R1);
        S[2] = S[2] + widen(R2);
    }
    double val = 0.0;
    if (valid) {
        const double2 nS = n[0] * S[0] + n[1] * S[1] + n[2] * S[2];
        double f2 = 0.0;
        for (int c = 0; c < 3; ++c) f2 += abs2_(S[c] - n[c] * nS);
        val = w * f2;
    }
    // block reduction (fixed order)
    __shared__ double red[FAR_THREADS / 32];
    for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = val;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int i = 0; i < FAR_THREADS / 32; ++i) a += red[i];
        part[(size_t)s * gridDim.x + blockIdx.x] = a;
    }
}

__global__ void k_far_sum(int S, int nb, const double* part, double* sums) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    double a = 0.0;
    for (int b = 0; b < nb; ++b) a += part[(size_t)s * nb + b];
    sums[s] = a;
}

template <typename Rl>
void launch_farfield(const LatticeDev& L, int S, const cx<Rl>* u, const double2* kappa_sys, const double* dirs,
                     const double* weights, int n_dir, double* part, double* sums, cudaStream_t st) {
    const int nb = (n_dir + FAR_THREADS - 1) / FAR_THREADS;
    const size_t sm = (size_t)FAR_CC * 3 * L.Nz * sizeof(cx<Rl>);
    count_launch();
    k_far<Rl><<<dim3(nb, S), FAR_THREADS, sm, st>>>(L, u, kappa_sys, dirs, weights, n_dir, part);
    count_launch();
    k_far_sum<<<(S + 127) / 128, 128, 0, st>>>(S, nb, part, sums);
}

void prepare_far_kernels() {
    cudaFuncSetAttribute(k_far<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_far<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

template void launch_farfield<float>(const LatticeDev&, int, const float2*, const double2*, const double*, const double*,
                                     int, double*, double*, cudaStream_t);
template void launch_farfield<double>(const LatticeDev&, int, const double2*, const double2*, const double*,
                                      const double*, int, double*, double*, cudaStream_t);

}  // namespace eels
