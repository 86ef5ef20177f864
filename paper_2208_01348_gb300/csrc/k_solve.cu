// Krylov iterations, FP64 refinement vectors and the loss reductions.
//
// QMR for complex-symmetric matrices (Freund, SIAM J. Sci. Stat. Comput. 13
// (1992) 425), the solver family the paper uses (Sec. S5).  The Lanczos
// process runs with the unconjugated bilinear form x^T y (the DDA matrix is
// complex symmetric, A = A^T) on unit-norm vectors:
//   w = A v_n,  alpha_n = v_n^T w / delta_n,  v~ = w - alpha_n v_n - beta_n v_{n-1},
//   rho_{n+1} = ||v~||,  v_{n+1} = v~ / rho_{n+1},  delta_{n+1} = v_{n+1}^T v_{n+1},
//   beta_{n+1} = rho_{n+1} delta_{n+1} / delta_n,
// and the quasi-residual ||rho_1 e_1 - H_n z|| is minimised with Givens
// rotations of the tridiagonal H_n (columns (beta_n, alpha_n, rho_{n+1})):
//   theta = s_{n-2} beta_n, eta = c_{n-1} c_{n-2} beta_n + s_{n-1} alpha_n,
//   mu = -conj(s_{n-1}) c_{n-2} beta_n + c_{n-1} alpha_n,
//   c_n = |mu| / r, s_n = (mu/|mu|) rho_{n+1} / r, r_n = (mu/|mu|) r,
//   r = sqrt(|mu|^2 + rho_{n+1}^2),  t_n = c_n tau_n,  tau_{n+1} = -conj(s_n) tau_n,
//   p_n = (v_n - eta p_{n-1} - theta p_{n-2}) / r_n,  x_n = x_{n-1} + t_n p_n.
// The iteration stops when |tau_{n+1}| <= eps ||b||.
//
// Every reduction is two-level and deterministic: a fixed grid of blocks
// per system (independent of how many systems share a launch) writes
// partial sums; consumers add them in block order.  Partial sums of FP32
// vectors are accumulated in FP32 inside a block.
#include <algorithm>

#include "solve.h"

namespace eels {

// --------------------------------------------------------------- reductions
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sums K values over the block; result valid in thread 0.
template <typename T, int K>
__device__ __forceinline__ void block_sum(T (&v)[K]) {
    __shared__ T sh[32 * K];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = warp_sum(v[k]);
    if (lane == 0)
        for (int k = 0; k < K; ++k) sh[wid * K + k] = v[k];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            T t = lane < nw ? sh[lane * K + k] : (T)0;
            v[k] = warp_sum(t);
        }
    }
    __syncthreads();
}

// part[s][blk][0..3] = (Re sum a.b, Im sum a.b, sum |a|^2, sum |b|^2)   (a.b unconjugated)
template <typename Rl>
__global__ void k_dot(int n3, int nblk, const cx<Rl>* __restrict__ a, const cx<Rl>* __restrict__ b, double* part,
                      const int* active) {
    const int s = blockIdx.y, blk = blockIdx.x;
    if (active && !active[s]) return;
    const size_t off = (size_t)s * n3;
    const int i0 = blk * RED_CHUNK, i1 = min(n3, i0 + RED_CHUNK);
    Rl v[4] = {0, 0, 0, 0};
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const cx<Rl> x = a[off + i], y = b[off + i];
        v[0] += x.x * y.x - x.y * y.y;
        v[1] += x.x * y.y + x.y * y.x;
        v[2] += x.x * x.x + x.y * x.y;
        v[3] += y.x * y.x + y.y * y.y;
    }
    block_sum<Rl, 4>(v);
    if (threadIdx.x == 0) {
        double* p = part + ((size_t)s * nblk + blk) * 4;
        p[0] = v[0]; p[1] = v[1]; p[2] = v[2]; p[3] = v[3];
    }
}

// Sums part[s][b][0..3] over the blocks b < nblk: lane l adds blocks l, l+32,
// ... in order, then a fixed shuffle tree adds the lanes.  Called by all 32
// lanes of a warp; every lane receives the sums.  The order depends only on
// nblk, so a system's result does not depend on the other systems.
__device__ __forceinline__ void warp_sum_parts(const double* part, int s, int nblk, double (&o)[4]) {
    const int lane = threadIdx.x & 31;
    const double2* p = reinterpret_cast<const double2*>(part + (size_t)s * nblk * 4);
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    for (int b = lane; b < nblk; b += 32) {
        const double2 u = p[2 * b], v = p[2 * b + 1];
        a0 += u.x; a1 += u.y; a2 += v.x; a3 += v.y;
    }
    o[0] = warp_sum(a0); o[1] = warp_sum(a1); o[2] = warp_sum(a2); o[3] = warp_sum(a3);
}

// Warp-per-system kernels: 4 systems per 128-thread block.
__device__ __forceinline__ int warp_system() { return blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); }
static inline unsigned warp_blocks(int S) { return (unsigned)((S + 3) / 4); }

// ------------------------------------------------------------------- QMR
template <typename Rl>
__global__ void k_qmr_start(KrylovArgs<Rl> k) {
    const int s = warp_system();
    if (s >= k.S) return;
    if (!k.active[s]) return;
    double o[4];
    warp_sum_parts(k.part_a, s, k.nblk, o);     // (b.b, |b|^2)
    if (threadIdx.x & 31) return;
    QmrState q;
    const double rho = sqrt(o[2]);
    q.bnorm = rho;
    q.beta = make_double2(0, 0);
    q.c1 = q.c2 = 1.0;
    q.s1 = q.s2 = make_double2(0, 0);
    q.tau = make_double2(rho, 0);
    q.iters = 0;
    q.qres = 1.0;
    q.eta = q.theta = q.t = make_double2(0, 0);
    q.rinv = make_double2(0, 0);
    if (rho > 0.0) {
        q.inv_rho = 1.0 / rho;
        q.delta = make_double2(o[0] / (rho * rho), o[1] / (rho * rho));
        q.status = 0;
    } else {                        // zero right-hand side: x = 0 is exact
        q.inv_rho = 0.0;
        q.delta = make_double2(1, 0);
        q.status = 1;
        q.qres = 0.0;
        k.active[s] = 0;
        atomicSub(k.n_active, 1);
    }
    k.qmr[s] = q;
}

// v_1 = b / rho_1; zero v_0, p slots and x
template <typename Rl>
__global__ void k_qmr_scale(KrylovArgs<Rl> k) {
    const int s = blockIdx.y;
    if (!k.active[s]) return;
    const Rl ir = (Rl)k.qmr[s].inv_rho;
    const size_t off = (size_t)s * k.n3;
    const cx<Rl> z = mk<cx<Rl>>(0.0, 0.0);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k.n3; i += gridDim.x * blockDim.x) {
        k.V[1][off + i] = ir * k.V[1][off + i];
        k.V[0][off + i] = z;
        k.P[0][off + i] = z; k.P[1][off + i] = z; k.P[2][off + i] = z;
        k.X[off + i] = z;
    }
}

// v~ = w - alpha v_n - beta_n v_{n-1}  (into W); partial sums of v~.v~ and |v~|^2
template <typename Rl>
__global__ void k_lanczos(KrylovArgs<Rl> k, int n) {
    const int s = blockIdx.y, blk = blockIdx.x;
    if (!k.active[s]) return;
    __shared__ double2 sc[2];
    if (threadIdx.x < 32) {
        double o[4];
        warp_sum_parts(k.part_a, s, k.nblk_a, o);
        if (threadIdx.x == 0) {
            const QmrState& q = k.qmr[s];
            sc[0] = cdiv(make_double2(o[0], o[1]), q.delta);
            sc[1] = q.beta;
        }
    }
    __syncthreads();
    const cx<Rl> al = cvt<cx<Rl>>(sc[0]), be = cvt<cx<Rl>>(sc[1]);
    const cx<Rl>* v = k.V[n & 1];
    const cx<Rl>* vp = k.V[(n + 1) & 1];
    const size_t off = (size_t)s * k.n3;
    const int i0 = blk * RED_CHUNK, i1 = min(k.n3, i0 + RED_CHUNK);
    Rl acc[4] = {0, 0, 0, 0};
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const cx<Rl> t = k.W[off + i] - al * v[off + i] - be * vp[off + i];
        k.W[off + i] = t;
        acc[0] += t.x * t.x - t.y * t.y;
        acc[1] += 2 * t.x * t.y;
        acc[2] += t.x * t.x + t.y * t.y;
    }
    block_sum<Rl, 4>(acc);
    if (threadIdx.x == 0) {
        double* p = k.part_b + ((size_t)s * k.nblk + blk) * 4;
        p[0] = acc[0]; p[1] = acc[1]; p[2] = acc[2]; p[3] = 0.0;
    }
}

template <typename Rl>
__global__ void k_qmr_step(KrylovArgs<Rl> k) {
    const int s = warp_system();
    if (s >= k.S) return;
    const bool lead = (threadIdx.x & 31) == 0;
    if (!k.active[s]) {
        if (lead) k.upd[s] = 0;
        return;
    }
    double oa[4], ob[4];
    warp_sum_parts(k.part_a, s, k.nblk_a, oa);
    warp_sum_parts(k.part_b, s, k.nblk, ob);
    if (!lead) return;
    QmrState q = k.qmr[s];
    // delta_1 = v_1^T v_1 / |v_1|^2 below the rounding floor of the vector
    // precision: the Lanczos process breaks down at its start (alpha_1 would be
    // divided by rounding noise and the rotated tau collapse to a false
    // convergence).  Stop with status 3 and the zero x that k_qmr_scale wrote.
    const double delta_floor = sizeof(Rl) == 4 ? 1e-5 : 1e-12;
    if (q.iters == 0 && !(cabs_(q.delta) >= delta_floor)) {
        q.iters = 1;
        q.status = 3;
        k.qmr[s] = q;
        k.upd[s] = 0;
        k.active[s] = 0;
        atomicSub(k.n_active, 1);
        return;
    }
    const double2 alpha = cdiv(make_double2(oa[0], oa[1]), q.delta);
    const double rho_n = sqrt(ob[2]);
    // Givens: apply rotations n-2, n-1 to the column (beta_n, alpha_n, rho_{n+1})
    const double2 theta = q.s2 * q.beta;
    const double2 tmp = q.c2 * q.beta;
    const double2 eta = q.c1 * tmp + q.s1 * alpha;
    const double2 mu = q.c1 * alpha - conj_(q.s1) * tmp;
    const double amu = cabs_(mu);
    double c;
    double2 sn, r;
    if (amu == 0.0) {
        c = 0.0; sn = make_double2(1, 0); r = make_double2(rho_n, 0);
    } else {
        const double ra = hypot(amu, rho_n);
        const double2 ph = (1.0 / amu) * mu;
        c = amu / ra; sn = (rho_n / ra) * ph; r = ra * ph;
    }
    q.theta = theta;
    q.eta = eta;
    q.rinv = cdiv(make_double2(1, 0), r);
    q.t = c * q.tau;
    q.tau = -(conj_(sn) * q.tau);
    q.c2 = q.c1; q.s2 = q.s1; q.c1 = c; q.s1 = sn;
    q.iters += 1;
    q.qres = cabs_(q.tau) / q.bnorm;
    int next = 1;
    if (rho_n > 0.0) {
        const double2 dn = make_double2(ob[0] / (rho_n * rho_n), ob[1] / (rho_n * rho_n));
        q.beta = cdiv(rho_n * dn, q.delta);
        q.inv_rho = 1.0 / rho_n;
        if (cabs_(dn) < 1e-30) { q.status = 3; next = 0; }
        q.delta = dn;
    } else {
        q.inv_rho = 0.0;           // invariant subspace reached: the update below is exact
        q.status = 1; next = 0;
    }
    if (next && q.qres <= (k.eps_sys ? k.eps_sys[s] : k.eps)) { q.status = 1; next = 0; }
    if (next && q.iters >= k.max_iter) { q.status = 2; next = 0; }
    if (!(q.qres == q.qres)) { q.status = 3; next = 0; }   // NaN guard
    k.qmr[s] = q;
    k.upd[s] = 1;                   // this iteration's vector update still applies
    if (!next) {                    // later kernels of the next iterations skip the system
        k.active[s] = 0;
        atomicSub(k.n_active, 1);
    }
}

// p_n = (v_n - eta p_{n-1} - theta p_{n-2}) / r_n ; x += t p_n ; v_{n+1} = v~ / rho_{n+1}
template <typename Rl>
__global__ void k_qmr_update(KrylovArgs<Rl> k, int n) {
    const int s = blockIdx.y;
    if (!k.upd[s]) return;
    using C = cx<Rl>;
    const QmrState& q = k.qmr[s];
    const C eta = cvt<C>(q.eta), th = cvt<C>(q.theta), ri = cvt<C>(q.rinv), t = cvt<C>(q.t);
    const Rl ir = (Rl)q.inv_rho;
    const C* v = k.V[n & 1];
    C* vn = k.V[(n + 1) & 1];
    C* pn = k.P[n % 3];
    const C* p1 = k.P[(n + 2) % 3];
    const C* p2 = k.P[(n + 1) % 3];
    const size_t off = (size_t)s * k.n3;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k.n3; i += gridDim.x * blockDim.x) {
        const C p = ri * (v[off + i] - eta * p1[off + i] - th * p2[off + i]);
        pn[off + i] = p;
        k.X[off + i] = k.X[off + i] + t * p;
        vn[off + i] = ir * k.W[off + i];
    }
}


// About four elements per thread and system: when only a few systems are
// still iterating, their vector passes still spread over the whole GPU.
static inline dim3 vec_grid(int n3, int S) {
    int bx = (n3 + 1023) / 1024;
    if (bx > 1024) bx = 1024;
    return dim3(bx, S);
}

template <typename Rl>
void launch_qmr_init(const KrylovArgs<Rl>& k, cudaStream_t st) {
    count_launch();
    k_dot<Rl><<<dim3(k.nblk, k.S), RED_THREADS, 0, st>>>(k.n3, k.nblk, k.V[1], k.V[1], k.part_a, k.active);
    count_launch();
    k_qmr_start<Rl><<<warp_blocks(k.S), 128, 0, st>>>(k);
    count_launch();
    k_qmr_scale<Rl><<<vec_grid(k.n3, k.S), 256, 0, st>>>(k);
}

template <typename Rl>
void launch_qmr_post_matvec(const KrylovArgs<Rl>& k, int n, bool dot_done, cudaStream_t st) {
    if (!dot_done) {
        count_launch();
        k_dot<Rl><<<dim3(k.nblk, k.S), RED_THREADS, 0, st>>>(k.n3, k.nblk, k.V[n & 1], k.W, k.part_a, k.active);
    }
    count_launch();
    k_lanczos<Rl><<<dim3(k.nblk, k.S), RED_THREADS, 0, st>>>(k, n);
    count_launch();
    k_qmr_step<Rl><<<warp_blocks(k.S), 128, 0, st>>>(k);
    count_launch();
    k_qmr_update<Rl><<<vec_grid(k.n3, k.S), 256, 0, st>>>(k, n);
}

template void launch_qmr_init<float>(const KrylovArgs<float>&, cudaStream_t);
template void launch_qmr_init<double>(const KrylovArgs<double>&, cudaStream_t);
template void launch_qmr_post_matvec<float>(const KrylovArgs<float>&, int, bool, cudaStream_t);
template void launch_qmr_post_matvec<double>(const KrylovArgs<double>&, int, bool, cudaStream_t);

// ------------------------------------------------------------------ QMR2
// QMR from coupled two-term recurrences (Freund & Nachtigal, SIAM J. Sci.
// Comput. 15 (1994) 313), the variant the paper found slightly faster than
// the three-term one (Sec. S5).  With A = A^T the left Lanczos sequence
// equals the right one, so an iteration costs one matvec.  Starting from
// v_1 = b / rho_1, p_1 = v_1, d_0 = 0, gamma_0 = 1, eta_0 = -1, tau_0 = ||b||:
//   eps_n = p_n^T (A p_n),  beta_n = eps_n / delta_n,
//   v~ = A p_n - beta_n v_n,  rho_{n+1} = ||v~||,  delta_{n+1} = v~^T v~ / rho_{n+1}^2,
//   theta_n = rho_{n+1} / (gamma_{n-1} |beta_n|),  gamma_n = (1 + theta_n^2)^(-1/2),
//   eta_n = -eta_{n-1} rho_n gamma_n^2 / (beta_n gamma_{n-1}^2),
//   d_n = eta_n p_n + (theta_{n-1} gamma_n)^2 d_{n-1},  x_n = x_{n-1} + d_n,
//   v_{n+1} = v~ / rho_{n+1},  p_{n+1} = v_{n+1} - (rho_{n+1} delta_{n+1} / eps_n) p_n,
// with the quasi-residual norm tau_n = tau_{n-1} theta_n gamma_n (the same
// quantity the three-term form minimises).  In exact arithmetic the iterates
// are those of the three-term form; in FP32 the two-term recurrences keep
// the Lanczos vectors biorthogonal far longer.
template <typename Rl>
__global__ void k_qmr2_start(KrylovArgs<Rl> k) {
    const int s = warp_system();
    if (s >= k.S) return;
    if (!k.active[s]) return;
    double o[4];
    warp_sum_parts(k.part_a, s, k.nblk, o);     // (b.b, |b|^2)
    if (threadIdx.x & 31) return;
    Qmr2State q;
    const double rho = sqrt(o[2]);
    q.bnorm = rho;
    q.rho = rho;
    q.tau = rho;
    q.gam = 1.0;
    q.th = 0.0;
    q.cd = 0.0;
    q.eta = make_double2(-1, 0);
    q.cp = make_double2(0, 0);
    q.iters = 0;
    q.qres = 1.0;
    q.status = 0;
    q.delta = make_double2(1, 0);
    q.inv_rho = 0.0;
    if (rho > 0.0) {
        q.inv_rho = 1.0 / rho;
        // v_1^T v_1 ~ 0 is caught by the first step, after k_qmr2_scale has
        // zeroed x (a system stopped here would keep a stale x)
        q.delta = make_double2(o[0] / (rho * rho), o[1] / (rho * rho));
    } else {                        // zero right-hand side: x = 0 is exact
        q.status = 1;
        q.qres = 0.0;
    }
    if (q.status != 0) {
        k.active[s] = 0;
        atomicSub(k.n_active, 1);
    }
    k.qmr2[s] = q;
}

// v_1 = b / rho_1 (in V[1]); p_1 = v_1; d_0 = 0; x = 0
template <typename Rl>
__global__ void k_qmr2_scale(KrylovArgs<Rl> k) {
    const int s = blockIdx.y;
    if (!k.active[s]) return;
    const Rl ir = (Rl)k.qmr2[s].inv_rho;
    const size_t off = (size_t)s * k.n3;
    const cx<Rl> z = mk<cx<Rl>>(0.0, 0.0);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k.n3; i += gridDim.x * blockDim.x) {
        const cx<Rl> v = ir * k.V[1][off + i];
        k.V[1][off + i] = v;
        k.P[0][off + i] = v;
        k.P[1][off + i] = z;
        k.X[off + i] = z;
    }
}

// v~ = A p_n - beta_n v_n (into W), beta_n = eps_n / delta_n with eps_n from
// part_a; partial sums of v~.v~ and |v~|^2 into part_b
template <typename Rl>
__global__ void k_qmr2_lanczos(KrylovArgs<Rl> k) {
    const int s = blockIdx.y, blk = blockIdx.x;
    if (!k.active[s]) return;
    __shared__ double2 sc;
    if (threadIdx.x < 32) {
        double o[4];
        warp_sum_parts(k.part_a, s, k.nblk_a, o);
        if (threadIdx.x == 0) sc = cdiv(make_double2(o[0], o[1]), k.qmr2[s].delta);
    }
    __syncthreads();
    const cx<Rl> be = cvt<cx<Rl>>(sc);
    const cx<Rl>* v = k.V[1];
    const size_t off = (size_t)s * k.n3;
    const int i0 = blk * RED_CHUNK, i1 = min(k.n3, i0 + RED_CHUNK);
    Rl acc[4] = {0, 0, 0, 0};
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const cx<Rl> t = k.W[off + i] - be * v[off + i];
        k.W[off + i] = t;
        acc[0] += t.x * t.x - t.y * t.y;
        acc[1] += 2 * t.x * t.y;
        acc[2] += t.x * t.x + t.y * t.y;
    }
    block_sum<Rl, 4>(acc);
    if (threadIdx.x == 0) {
        double* p = k.part_b + ((size_t)s * k.nblk + blk) * 4;
        p[0] = acc[0]; p[1] = acc[1]; p[2] = acc[2]; p[3] = 0.0;
    }
}

template <typename Rl>
__global__ void k_qmr2_step(KrylovArgs<Rl> k) {
    const int s = warp_system();
    if (s >= k.S) return;
    const bool lead = (threadIdx.x & 31) == 0;
    if (!k.active[s]) {
        if (lead) k.upd[s] = 0;
        return;
    }
    double oa[4], ob[4];
    warp_sum_parts(k.part_a, s, k.nblk_a, oa);
    warp_sum_parts(k.part_b, s, k.nblk, ob);
    if (!lead) return;
    Qmr2State q = k.qmr2[s];
    // delta_1 = v_1^T v_1 / |v_1|^2 below the rounding floor of the vector
    // precision: the Lanczos process breaks down at its start (beta_1 would be
    // eps_1 / rounding noise, and tau collapse to a false convergence with
    // x ~ 0).  Stop with status 3 and the zero x that k_qmr2_scale wrote.
    const double delta_floor = sizeof(Rl) == 4 ? 1e-5 : 1e-12;
    if (q.iters == 0 && !(cabs_(q.delta) >= delta_floor)) {
        q.iters = 1;
        q.status = 3;
        k.qmr2[s] = q;
        k.upd[s] = 0;
        k.active[s] = 0;
        atomicSub(k.n_active, 1);
        return;
    }
    const double2 eps = make_double2(oa[0], oa[1]);
    const double2 beta = cdiv(eps, q.delta);
    const double abeta = cabs_(beta);
    const double rho_n = sqrt(ob[2]);
    q.iters += 1;
    int next = 1, upd = 1;
    if (!(abeta > 0.0) || !(rho_n == rho_n)) {
        // eps_n = 0 (or not finite): the coupled recurrences break down and
        // this iteration's update is undefined; x keeps its previous value
        q.status = 3; next = 0; upd = 0;
    } else {
        const double th = rho_n / (q.gam * abeta);
        const double g = 1.0 / sqrt(1.0 + th * th);
        const double f = q.rho * g * g / (q.gam * q.gam);
        q.eta = -(f * cdiv(q.eta, beta));
        q.cd = (q.th * g) * (q.th * g);
        q.tau = q.tau * th * g;
        q.qres = q.tau / q.bnorm;
        q.th = th;
        q.gam = g;
        if (rho_n > 0.0) {
            const double2 dn = make_double2(ob[0] / (rho_n * rho_n), ob[1] / (rho_n * rho_n));
            q.cp = cdiv(rho_n * dn, eps);
            q.inv_rho = 1.0 / rho_n;
            q.rho = rho_n;
            if (!(cabs_(dn) >= 1e-30)) { q.status = 3; next = 0; }
            q.delta = dn;
        } else {                    // invariant subspace reached: the update below is exact
            q.cp = make_double2(0, 0);
            q.inv_rho = 0.0;
            q.status = 1; next = 0;
        }
        if (next && q.qres <= (k.eps_sys ? k.eps_sys[s] : k.eps)) { q.status = 1; next = 0; }
        if (next && q.iters >= k.max_iter) { q.status = 2; next = 0; }
        if (!(q.qres == q.qres) || !(q.eta.x == q.eta.x) || !(q.eta.y == q.eta.y)) {   // NaN guard
            q.status = 3; next = 0; upd = 0;
        }
    }
    k.qmr2[s] = q;
    k.upd[s] = upd;
    if (!next) {
        k.active[s] = 0;
        atomicSub(k.n_active, 1);
    }
}

// d_n = eta_n p_n + cd d_{n-1}; x += d_n; v_{n+1} = v~ / rho_{n+1};
// p_{n+1} = v_{n+1} - cp p_n
template <typename Rl>
__global__ void k_qmr2_update(KrylovArgs<Rl> k) {
    const int s = blockIdx.y;
    if (!k.upd[s]) return;
    using C = cx<Rl>;
    const Qmr2State& q = k.qmr2[s];
    const C eta = cvt<C>(q.eta), cp = cvt<C>(q.cp);
    const Rl cd = (Rl)q.cd, ir = (Rl)q.inv_rho;
    const size_t off = (size_t)s * k.n3;
    C* v = k.V[1];
    C* p = k.P[0];
    C* d = k.P[1];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k.n3; i += gridDim.x * blockDim.x) {
        const C pn = p[off + i];
        const C dn = eta * pn + cd * d[off + i];
        d[off + i] = dn;
        k.X[off + i] = k.X[off + i] + dn;
        const C vn = ir * k.W[off + i];
        v[off + i] = vn;
        p[off + i] = vn - cp * pn;
    }
}

template <typename Rl>
void launch_qmr2_init(const KrylovArgs<Rl>& k, cudaStream_t st) {
    count_launch();
    k_dot<Rl><<<dim3(k.nblk, k.S), RED_THREADS, 0, st>>>(k.n3, k.nblk, k.V[1], k.V[1], k.part_a, k.active);
    count_launch();
    k_qmr2_start<Rl><<<warp_blocks(k.S), 128, 0, st>>>(k);
    count_launch();
    k_qmr2_scale<Rl><<<vec_grid(k.n3, k.S), 256, 0, st>>>(k);
}

template <typename Rl>
void launch_qmr2_post_matvec(const KrylovArgs<Rl>& k, bool dot_done, cudaStream_t st) {
    if (!dot_done) {
        count_launch();
        k_dot<Rl><<<dim3(k.nblk, k.S), RED_THREADS, 0, st>>>(k.n3, k.nblk, k.P[0], k.W, k.part_a, k.active);
    }
    count_launch();
    k_qmr2_lanczos<Rl><<<dim3(k.nblk, k.S), RED_THREADS, 0, st>>>(k);
    count_launch();
    k_qmr2_step<Rl><<<warp_blocks(k.S), 128, 0, st>>>(k);
    count_launch();
    k_qmr2_update<Rl><<<vec_grid(k.n3, k.S), 256, 0, st>>>(k);
}

template void launch_qmr2_init<float>(const KrylovArgs<float>&, cudaStream_t);
template void launch_qmr2_init<double>(const KrylovArgs<double>&, cudaStream_t);
template void launch_qmr2_post_matvec<float>(const KrylovArgs<float>&, bool, cudaStream_t);
template void launch_qmr2_post_matvec<double>(const KrylovArgs<double>&, bool, cudaStream_t);

// One thread: the chunk count bounds the loop whatever the systems do.
__global__ void k_loop_ctl(cudaGraphConditionalHandle h, const int* n_active, int* chunks, int max_chunks) {
    const int n = *chunks + 1;
    *chunks = n;
    cudaGraphSetConditional(h, (*n_active > 0 && n < max_chunks) ? 1u : 0u);
}

void launch_loop_ctl(cudaGraphConditionalHandle h, const int* n_active, int* chunks, int max_chunks, cudaStream_t st) {
    count_launch();
    k_loop_ctl<<<1, 1, 0, st>>>(h, n_active, chunks, max_chunks);
}

// ------------------------------------------------------------- BiCGStab
// van der Vorst (SIAM J. Sci. Stat. Comput. 13 (1992) 631) for a general
// complex matrix: shadow residual r^ = r0 and the conjugated inner product
// throughout, so rho_0 = ||r0||^2 > 0 and the method cannot break down at the
// start on a residual whose unconjugated square r^T r is near zero (where
// the complex-symmetric Lanczos process of QMR does).  Per iteration:
//   v = A p, alpha = rho / r^^H v, s = r - alpha v, t = A s,
//   omega = (t^H s) / (t^H t), x += alpha p + omega s, r = s - omega t,
//   rho' = r^^H r, beta = (rho'/rho)(alpha/omega), p = r + beta (p - omega v).

// part[s][blk] = (Re sum conj(a) b, Im, sum |a|^2, 0)
template <typename Rl>
__global__ void k_dotc(int n3, int nblk, const cx<Rl>* __restrict__ a, const cx<Rl>* __restrict__ b, double* part,
                       const int* active) {
    const int s = blockIdx.y, blk = blockIdx.x;
    if (active && !active[s]) return;
    const size_t off = (size_t)s * n3;
    const int i0 = blk * RED_CHUNK, i1 = min(n3, i0 + RED_CHUNK);
    Rl v[4] = {0, 0, 0, 0};
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const cx<Rl> x = a[off + i], y = b[off + i];
        v[0] += x.x * y.x + x.y * y.y;
        v[1] += x.x * y.y - x.y * y.x;
        v[2] += x.x * x.x + x.y * x.y;
    }
    block_sum<Rl, 4>(v);
    if (threadIdx.x == 0) {
        double* p = part + ((size_t)s * nblk + blk) * 4;
        p[0] = v[0]; p[1] = v[1]; p[2] = v[2]; p[3] = 0.0;
    }
}

// r^ = r, p = r, x = 0
template <typename Rl>
__global__ void k_bicg_copy(KrylovArgs<Rl> k) {
    const int s = blockIdx.y;
    if (!k.active[s]) return;
    const size_t off = (size_t)s * k.n3;
    const cx<Rl> z = mk<cx<Rl>>(0.0, 0.0);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k.n3; i += gridDim.x * blockDim.x) {
        const cx<Rl> r = k.R[off + i];
        k.Rh[off + i] = r;
        k.Pb[off + i] = r;
        k.X[off + i] = z;
    }
}

template <typename Rl>
__global__ void k_bicg_start(KrylovArgs<Rl> k) {
    const int s = warp_system();
    if (s >= k.S || !k.active[s]) return;
    double o[4];
    warp_sum_parts(k.part_a, s, k.nblk, o);     // (r^H r, |r|^2)
    if (threadIdx.x & 31) return;
    BicgState b;
    b.rho = make_double2(o[0], o[1]);
    b.bnorm = sqrt(o[2]);
    b.alpha = b.omega = b.beta = make_double2(0, 0);
    b.res = 1.0;
    b.iters = 0;
    b.status = 0;
    if (!(b.bnorm > 0.0)) {       // zero right-hand side: x = 0 is exact
        b.status = 1;
        b.res = 0.0;
        k.active[s] = 0;
        atomicSub(k.n_active, 1);
    }
    k.bicg[s] = b;
}

// alpha = rho / r^T v ; s = r - alpha v (into R)
template <typename Rl>
__global__ void k_bicg_s(KrylovArgs<Rl> k) {
    const int s = blockIdx.y;
    if (!k.active[s]) return;
    __shared__ double2 al;
    if (threadIdx.x < 32) {
        double o[4];
        warp_sum_parts(k.part_a, s, k.nblk, o);
        if (threadIdx.x == 0) {
            const double2 rv = make_double2(o[0], o[1]);
            al = (abs2_(rv) > 0.0) ? cdiv(k.bicg[s].rho, rv) : make_double2(0, 0);
            if (blockIdx.x == 0) k.bicg[s].alpha = al;
        }
    }
    __syncthreads();
    const cx<Rl> a = cvt<cx<Rl>>(al);
    const size_t off = (size_t)s * k.n3;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k.n3; i += gridDim.x * blockDim.x)
        k.R[off + i] = k.R[off + i] - a * k.Vb[off + i];
}

// omega = t^H s / t^H t ; x += alpha p + omega s ; r = s - omega t ; partials of r^.r and |r|^2
template <typename Rl>
__global__ void k_bicg_x(KrylovArgs<Rl> k) {
    const int s = blockIdx.y, blk = blockIdx.x;
    if (!k.active[s]) return;
    __shared__ double2 sc[2];
    if (threadIdx.x < 32) {
        double o[4];
        warp_sum_parts(k.part_b, s, k.nblk, o);
        if (threadIdx.x == 0) {
            sc[0] = k.bicg[s].alpha;
            sc[1] = o[2] > 0.0 ? make_double2(o[0] / o[2], o[1] / o[2]) : make_double2(0, 0);
            if (blk == 0) k.bicg[s].omega = sc[1];
        }
    }
    __syncthreads();
    const cx<Rl> al = cvt<cx<Rl>>(sc[0]), om = cvt<cx<Rl>>(sc[1]);
    const size_t off = (size_t)s * k.n3;
    const int i0 = blk * RED_CHUNK, i1 = min(k.n3, i0 + RED_CHUNK);
    Rl acc[4] = {0, 0, 0, 0};
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const cx<Rl> sv = k.R[off + i];
        k.X[off + i] = k.X[off + i] + al * k.Pb[off + i] + om * sv;
        const cx<Rl> r = sv - om * k.Tb[off + i];
        k.R[off + i] = r;
        const cx<Rl> h = k.Rh[off + i];
        acc[0] += h.x * r.x + h.y * r.y;      // conj(r^) . r
        acc[1] += h.x * r.y - h.y * r.x;
        acc[2] += r.x * r.x + r.y * r.y;
    }
    block_sum<Rl, 4>(acc);
    if (threadIdx.x == 0) {
        double* p = k.part_a + ((size_t)s * k.nblk + blk) * 4;
        p[0] = acc[0]; p[1] = acc[1]; p[2] = acc[2]; p[3] = 0.0;
    }
}

template <typename Rl>
__global__ void k_bicg_step(KrylovArgs<Rl> k) {
    const int s = warp_system();
    if (s >= k.S) return;
    const bool lead = (threadIdx.x & 31) == 0;
    if (!k.active[s]) {
        if (lead) k.upd[s] = 0;
        return;
    }
    double o[4];
    warp_sum_parts(k.part_a, s, k.nblk, o);
    if (!lead) return;
    BicgState b = k.bicg[s];
    const double2 rho_n = make_double2(o[0], o[1]);
    b.res = sqrt(o[2]) / b.bnorm;
    b.iters += 1;
    int next = 1;
    const double eps = k.eps_sys ? k.eps_sys[s] : k.eps;
    if (b.res <= eps) { b.status = 1; next = 0; }
    else if (b.iters >= k.max_iter) { b.status = 2; next = 0; }
    else if (!(abs2_(b.omega) > 0.0) || !(abs2_(b.rho) > 0.0) || !(b.res == b.res)) { b.status = 3; next = 0; }
    if (next) {
        b.beta = cdiv(rho_n, b.rho) * cdiv(b.alpha, b.omega);
        b.rho = rho_n;
    }
    k.bicg[s] = b;
    k.upd[s] = next;
    if (!next) {
        k.active[s] = 0;
        atomicSub(k.n_active, 1);
    }
}

// p = r + beta (p - omega v)
template <typename Rl>
__global__ void k_bicg_p(KrylovArgs<Rl> k) {
    const int s = blockIdx.y;
    if (!k.upd[s]) return;
    const cx<Rl> be = cvt<cx<Rl>>(k.bicg[s].beta), om = cvt<cx<Rl>>(k.bicg[s].omega);
    const size_t off = (size_t)s * k.n3;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k.n3; i += gridDim.x * blockDim.x)
        k.Pb[off + i] = k.R[off + i] + be * (k.Pb[off + i] - om * k.Vb[off + i]);
}

template <typename Rl>
void launch_bicg_init(const KrylovArgs<Rl>& k, cudaStream_t st) {
    count_launch();
    k_bicg_copy<Rl><<<vec_grid(k.n3, k.S), 256, 0, st>>>(k);
    count_launch();
    k_dotc<Rl><<<dim3(k.nblk, k.S), RED_THREADS, 0, st>>>(k.n3, k.nblk, k.R, k.R, k.part_a, k.active);
    count_launch();
    k_bicg_start<Rl><<<warp_blocks(k.S), 128, 0, st>>>(k);
}

template <typename Rl>
void launch_bicg_stage1(const KrylovArgs<Rl>& k, cudaStream_t st) {
    count_launch();
    k_dotc<Rl><<<dim3(k.nblk, k.S), RED_THREADS, 0, st>>>(k.n3, k.nblk, k.Rh, k.Vb, k.part_a, k.active);
    count_launch();
    k_bicg_s<Rl><<<vec_grid(k.n3, k.S), 256, 0, st>>>(k);
}

template <typename Rl>
void launch_bicg_stage2(const KrylovArgs<Rl>& k, cudaStream_t st) {
    count_launch();
    k_dotc<Rl><<<dim3(k.nblk, k.S), RED_THREADS, 0, st>>>(k.n3, k.nblk, k.Tb, k.R, k.part_b, k.active);
    count_launch();
    k_bicg_x<Rl><<<dim3(k.nblk, k.S), RED_THREADS, 0, st>>>(k);
    count_launch();
    k_bicg_step<Rl><<<warp_blocks(k.S), 128, 0, st>>>(k);
    count_launch();
    k_bicg_p<Rl><<<vec_grid(k.n3, k.S), 256, 0, st>>>(k);
}

template void launch_bicg_init<float>(const KrylovArgs<float>&, cudaStream_t);
template void launch_bicg_init<double>(const KrylovArgs<double>&, cudaStream_t);
template void launch_bicg_stage1<float>(const KrylovArgs<float>&, cudaStream_t);
template void launch_bicg_stage1<double>(const KrylovArgs<double>&, cudaStream_t);
template void launch_bicg_stage2<float>(const KrylovArgs<float>&, cudaStream_t);
template void launch_bicg_stage2<double>(const KrylovArgs<double>&, cudaStream_t);


// ------------------------------------------------------- FP64 refinement
__global__ void k_rhs_init(LatticeDev L, int S, const double2* e, const double2* coef, double2* b, double2* x, double2* r) {
    const int s = blockIdx.y;
    const size_t n3 = (size_t)3 * L.N, off = (size_t)s * n3;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (size_t)gridDim.x * blockDim.x) {
        const int dip = (int)(i % L.N);
        const double2 v = coef[(size_t)s * EELS_MAX_MAT + L.mat[dip]] * e[off + i];
        b[off + i] = v;
        r[off + i] = v;
        x[off + i] = make_double2(0, 0);
    }
}

__global__ void k_norms2(int n3, int nblk, const double2* a, const double2* b, double* part) {
    const int s = blockIdx.y, blk = blockIdx.x;
    const size_t off = (size_t)s * n3;
    const int i0 = blk * RED_CHUNK, i1 = min(n3, i0 + RED_CHUNK);
    double v[2] = {0, 0};
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        v[0] += abs2_(a[off + i]);
        v[1] += abs2_(b[off + i]);
    }
    block_sum<double, 2>(v);
    if (threadIdx.x == 0) {
        double* p = part + ((size_t)s * nblk + blk) * 4;
        p[0] = v[0]; p[1] = v[1]; p[2] = 0; p[3] = 0;
    }
}

__global__ void k_residual_check(int S, int nblk, const double* part, double eps, double eps_floor, double safety,
                                 double* res, double* rnorm, int* outer, int* n_outer, double* eps_sys) {
    const int s = warp_system();
    if (s >= S) return;
    double o[4];
    warp_sum_parts(part, s, nblk, o);
    if (threadIdx.x & 31) return;
    const double rn = sqrt(o[0]), bn = sqrt(o[1]);
    const double r = bn > 0 ? rn / bn : 0.0;
    res[s] = r;
    rnorm[s] = rn;
    const int go = (r > eps) && (rn > 0.0) && (r == r);
    outer[s] = go;
    if (eps_sys) eps_sys[s] = go ? fmin(1e-2, fmax(eps_floor, safety * eps / r)) : 1.0;
    if (go) atomicAdd(n_outer, 1);
}

template <typename Rl>
__global__ void k_make_inner_rhs(int S, int n3, const double2* r, const double* rnorm, const int* outer, cx<Rl>* v,
                                 int* active, int* n_active) {
    const int s = blockIdx.y;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        active[s] = outer[s];
        if (outer[s]) atomicAdd(n_active, 1);
    }
    if (!outer[s]) return;
    const double ir = 1.0 / rnorm[s];
    const size_t off = (size_t)s * n3;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += gridDim.x * blockDim.x)
        v[off + i] = cvt<cx<Rl>>(ir * r[off + i]);
}

template <typename Rl>
__global__ void k_accumulate(int S, int n3, const cx<Rl>* xi, const double* rnorm, const int* outer, double2* x) {
    const int s = blockIdx.y;
    if (!outer[s]) return;
    const double rn = rnorm[s];
    const size_t off = (size_t)s * n3;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += gridDim.x * blockDim.x)
        x[off + i] = x[off + i] + rn * widen(xi[off + i]);
}

__global__ void k_sub(size_t n, const double2* b, const double2* y, double2* r) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        r[i] = b[i] - y[i];
}

__global__ void k_to_f32(size_t n, const double2* a, float2* b) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        b[i] = to_f(a[i]);
}

void launch_rhs_init(const LatticeDev& L, int S, const double2* e, const double2* coef, double2* b, double2* x,
                     double2* r, cudaStream_t st) {
    count_launch();
    k_rhs_init<<<vec_grid(3 * L.N, S), 256, 0, st>>>(L, S, e, coef, b, x, r);
}
void launch_norms2(int S, int n3, int nblk, const double2* a, const double2* b, double* part, cudaStream_t st) {
    count_launch();
    k_norms2<<<dim3(nblk, S), RED_THREADS, 0, st>>>(n3, nblk, a, b, part);
}
void launch_residual_check(int S, int nblk, const double* part, double eps, double eps_floor, double safety,
                           double* res, double* rnorm, int* outer, int* n_outer, double* eps_sys, cudaStream_t st) {
    cudaMemsetAsync(n_outer, 0, sizeof(int), st);
    count_launch();
    k_residual_check<<<warp_blocks(S), 128, 0, st>>>(S, nblk, part, eps, eps_floor, safety, res, rnorm, outer, n_outer,
                                                      eps_sys);
}
template <typename Rl>
void launch_make_inner_rhs(int S, int n3, const double2* r, const double* rnorm, const int* outer, cx<Rl>* v,
                           int* active, int* n_active, cudaStream_t st) {
    cudaMemsetAsync(n_active, 0, sizeof(int), st);
    count_launch();
    k_make_inner_rhs<Rl><<<vec_grid(n3, S), 256, 0, st>>>(S, n3, r, rnorm, outer, v, active, n_active);
}
template <typename Rl>
void launch_accumulate(int S, int n3, const cx<Rl>* xi, const double* rnorm, const int* outer, double2* x,
                       cudaStream_t st) {
    count_launch();
    k_accumulate<Rl><<<vec_grid(n3, S), 256, 0, st>>>(S, n3, xi, rnorm, outer, x);
}
template void launch_make_inner_rhs<float>(int, int, const double2*, const double*, const int*, float2*, int*, int*, cudaStream_t);
template void launch_make_inner_rhs<double>(int, int, const double2*, const double*, const int*, double2*, int*, int*, cudaStream_t);
template void launch_accumulate<float>(int, int, const float2*, const double*, const int*, double2*, cudaStream_t);
template void launch_accumulate<double>(int, int, const double2*, const double*, const int*, double2*, cudaStream_t);

void launch_sub(int S, int n3, const double2* b, const double2* y, double2* r, cudaStream_t st) {
    const size_t n = (size_t)S * n3;
    count_launch();
    k_sub<<<(unsigned)std::min<size_t>((n + 255) / 256, 8192), 256, 0, st>>>(n, b, y, r);
}
void launch_to_f32(size_t n, const double2* a, float2* b, cudaStream_t st) {
    count_launch();
    k_to_f32<<<(unsigned)std::min<size_t>((n + 255) / 256, 8192), 256, 0, st>>>(n, a, b);
}

// ------------------------------------------------------------ losses
// Per block partial sums over dipoles: sum E_a.u (3 comps), sum conj(E).u, sum |u|^2 w.
// E_a = (-E_x, -E_y, E_z) exp(-2 i w (z - z0)/v)   (Eq. 34, second form)
__global__ void k_losses(LatticeDev L, const double2* e, const double2* x, const double2* coef, const double* wabs,
                         const double* wdv, const SysField* sys, double* part, int nblk) {
    const int s = blockIdx.y, blk = blockIdx.x;
    const size_t N = (size_t)L.N, off = (size_t)s * 3 * N;
    const int chunk = (L.N + nblk - 1) / nblk;
    const int i0 = blk * chunk, i1 = min(L.N, i0 + chunk);
    const double w = wdv[s];
    double v[5] = {0, 0, 0, 0, 0};
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const int m = L.mat[i];
        const double2 cf = coef[(size_t)s * EELS_MAX_MAT + m];
        const double2 ux = cf * x[off + i], uy = cf * x[off + N + i], uz = cf * x[off + 2 * N + i];
        const double2 ex = e[off + i], ey = e[off + N + i], ez = e[off + 2 * N + i];
        const int cell = L.dip_cell[i];
        const int iz = cell / (L.Nx * L.Ny);
        double2 ea;
        if (sys[s].along_z) {
            const double zr = (iz + 0.5) - 0.5 * L.Nz;
            double sn, cs;
            sincos(-2.0 * w * zr, &sn, &cs);
            const double2 ph = make_double2(cs, sn);
            ea = ph * (ez * uz - ex * ux - ey * uy);
        } else {   // E_a . u = exp(-2 i w z'/v) (2 (E.n)(n.u) - E.u)
            const SysField& p = sys[s];
            const int ix = cell % L.Nx, iy = (cell / L.Nx) % L.Ny;
            const double zp = ((ix + 0.5) - 0.5 * L.Nx - p.px) * p.nx + ((iy + 0.5) - 0.5 * L.Ny - p.py) * p.ny +
                              ((iz + 0.5) - 0.5 * L.Nz - p.pz) * p.nz;
            double sn, cs;
            sincos(-2.0 * w * zp, &sn, &cs);
            const double2 ph = make_double2(cs, sn);
            const double2 en = p.nx * ex + p.ny * ey + p.nz * ez, un = p.nx * ux + p.ny * uy + p.nz * uz;
            ea = ph * (2.0 * (en * un) - (ex * ux + ey * uy + ez * uz));
        }
        const double2 ec = conj_(ex) * ux + conj_(ey) * uy + conj_(ez) * uz;
        v[0] += ea.x; v[1] += ea.y; v[2] += ec.x; v[3] += ec.y;
        v[4] += (abs2_(ux) + abs2_(uy) + abs2_(uz)) * wabs[(size_t)s * EELS_MAX_MAT + m];
    }
    block_sum<double, 5>(v);
    if (threadIdx.x == 0) {
        double* p = part + ((size_t)s * nblk + blk) * 8;
        for (int q = 0; q < 5; ++q) p[q] = v[q];
    }
}

__global__ void k_sum_parts(int S, int nblk, int stride, int nval, const double* part, double* out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    for (int q = 0; q < nval; ++q) {
        double a = 0.0;
        for (int b = 0; b < nblk; ++b) a += part[((size_t)s * nblk + b) * stride + q];
        out[(size_t)s * nval + q] = a;
    }
}

void launch_losses(const LatticeDev& L, int S, const double2* e, const double2* x, const double2* coef,
                   const double* wabs, const double* wdv, const SysField* sys, double* part, int nblk, double* sums,
                   cudaStream_t st) {
    count_launch();
    k_losses<<<dim3(nblk, S), 256, 0, st>>>(L, e, x, coef, wabs, wdv, sys, part, nblk);
    count_launch();
    k_sum_parts<<<(S + 127) / 128, 128, 0, st>>>(S, nblk, 8, 5, part, sums);
}

__global__ void k_scaled_dipoles(LatticeDev L, int S, const double2* x, const double2* coef, double2* u64, float2* u32) {
    const int s = blockIdx.y;
    const size_t n3 = (size_t)3 * L.N, off = (size_t)s * n3;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (size_t)gridDim.x * blockDim.x) {
        const double2 u = coef[(size_t)s * EELS_MAX_MAT + L.mat[i % L.N]] * x[off + i];
        if (u64) u64[off + i] = u;
        if (u32) u32[off + i] = to_f(u);
    }
}
void launch_scaled_dipoles(const LatticeDev& L, int S, const double2* x, const double2* coef, double2* u64, float2* u32,
                           cudaStream_t st) {
    count_launch();
    k_scaled_dipoles<<<vec_grid(3 * L.N, S), 256, 0, st>>>(L, S, x, coef, u64, u32);
}

}  // namespace eels
