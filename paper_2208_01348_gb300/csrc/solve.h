// Krylov / refinement / loss kernels: launch interface.
#pragma once
#include "kernels.h"

namespace eels {

// Per-system scalars of the complex-symmetric QMR iteration (FP64).
struct QmrState {
    double2 delta;        // delta_n = v_n^T v_n (unconjugated)
    double2 beta;         // beta_n, coefficient of v_{n-1} in the Lanczos recurrence
    double2 s1, s2;       // Givens sines of rotations n-1, n-2
    double c1, c2;        // Givens cosines
    double2 tau;          // rotated right-hand side entry tau_n
    double2 eta, theta;   // p_n = (v_n - eta p_{n-1} - theta p_{n-2}) / r_n
    double2 rinv;         // 1 / r_n
    double2 t;            // x_n = x_{n-1} + t p_n
    double inv_rho;       // 1 / rho_{n+1}: v_{n+1} = v~_{n+1} / rho_{n+1}
    double bnorm;         // ||b||
    double qres;          // |tau_{n+1}| / ||b||
    int iters;
    int status;           // 0 running, 1 converged, 2 iteration limit, 3 breakdown
};

// Per-system scalars of QMR from coupled two-term recurrences (FP64).
struct Qmr2State {
    double2 delta;        // delta_n = v_n^T v_n (unconjugated)
    double2 eta;          // d_n = eta_n p_n + cd d_{n-1}
    double2 cp;           // p_{n+1} = v_{n+1} - cp p_n
    double rho;           // rho_n = ||v~_n||
    double gam, th;       // gamma_{n-1}, theta_{n-1}
    double cd;            // (theta_{n-1} gamma_n)^2
    double tau;           // quasi-residual norm tau_n
    double inv_rho;       // 1 / rho_{n+1}: v_{n+1} = v~_{n+1} / rho_{n+1}
    double bnorm;         // ||b||
    double qres;          // tau_n / ||b||
    int iters;
    int status;           // 0 running, 1 converged, 2 iteration limit, 3 breakdown
};
static_assert(sizeof(Qmr2State) <= sizeof(QmrState), "Qmr2State shares the QmrState buffer");

// BiCGStab per-system scalars (FP64).
struct BicgState {
    double2 rho, alpha, omega, beta;
    double bnorm, res;
    int iters, status;
};

template <typename Rl>
struct KrylovArgs {
    int S, n3, nblk;               // systems, vector length 3N, reduction blocks per system
    int nblk_a;                    // partial sums of v^T (A v) per system in part_a (3 Nx when the matvec writes them)
    cx<Rl>* V[2];                  // Lanczos vectors (slot n % 2 holds v_n)
    cx<Rl>* P[3];                  // QMR directions (slot n % 3 holds p_n)
    cx<Rl>* W;                     // A v_n, then v~_{n+1}
    cx<Rl>* X;                     // iterate
    // BiCGStab work vectors (R = residual, Rh = shadow, Pb, Vb, Sb, Tb)
    cx<Rl>* R; cx<Rl>* Rh; cx<Rl>* Pb; cx<Rl>* Vb; cx<Rl>* Sb; cx<Rl>* Tb;
    double* part_a;                // [S][nblk][4] block partial sums
    double* part_b;
    QmrState* qmr;
    Qmr2State* qmr2;               // same memory as qmr (one solver runs at a time)
    BicgState* bicg;
    int* active;                   // [S] 1 while the system iterates
    int* upd;                      // [S] 1 if this iteration's vector update applies
    int* n_active;                 // device counter of active systems
    double eps;                    // stop when the (quasi-)residual <= eps ||b||
    const double* eps_sys;         // per-system eps (overrides eps when non-null)
    int max_iter;
};

constexpr int RED_THREADS = 256;
constexpr int RED_CHUNK = 4096;    // vector entries per reduction block

// QMR (complex symmetric, Freund 1992): start from the rhs stored in V[1].
template <typename Rl> void launch_qmr_init(const KrylovArgs<Rl>& k, cudaStream_t st);
// One QMR iteration n >= 1; the caller supplies the matvec (W = A V[n%2]).
template <typename Rl> void launch_qmr_post_matvec(const KrylovArgs<Rl>& k, int n, bool dot_done, cudaStream_t st);
// QMR from coupled two-term recurrences (Freund & Nachtigal 1994), complex
// symmetric: rhs in V[1]; vector roles V[1] = v_n, P[0] = p_n (the matvec
// input, W = A P[0]), P[1] = d_n, X.
template <typename Rl> void launch_qmr2_init(const KrylovArgs<Rl>& k, cudaStream_t st);
template <typename Rl> void launch_qmr2_post_matvec(const KrylovArgs<Rl>& k, bool dot_done, cudaStream_t st);
// BiCGStab (van der Vorst 1992) with the shadow residual r^ = r0 and the
// conjugated inner product (general complex form); rhs in R, X = 0.
// Vector roles: R (residual; the rhs on entry, S = R - alpha V overwrites
// it), Rh (shadow), Pb (direction), Vb = A Pb, Tb = A S, X (iterate).
template <typename Rl> void launch_bicg_init(const KrylovArgs<Rl>& k, cudaStream_t st);
template <typename Rl> void launch_bicg_stage1(const KrylovArgs<Rl>& k, cudaStream_t st);   // after Vb = A Pb
template <typename Rl> void launch_bicg_stage2(const KrylovArgs<Rl>& k, cudaStream_t st);   // after Tb = A S

// Loop control of a captured inner solve (the last node of the body of a
// graph WHILE node): counts the chunk in *chunks and keeps the loop going
// while any system is active and fewer than max_chunks chunks have run.
void launch_loop_ctl(cudaGraphConditionalHandle h, const int* n_active, int* chunks, int max_chunks, cudaStream_t st);

// ---- FP64 refinement helpers (vectors [S][n3]) ----
// b = coef[mat] * e; x = 0; r = b
void launch_rhs_init(const LatticeDev& L, int S, const double2* e, const double2* coef, double2* b, double2* x,
                     double2* r, cudaStream_t st);
// part[s][blk] = (sum |a|^2, sum |b|^2)
void launch_norms2(int S, int n3, int nblk, const double2* a, const double2* b, double* part, cudaStream_t st);
// per system: rn = ||r||, res = rn / ||b||; outer[s] = res > eps; rnorm[s] = rn;
// eps_sys[s] = min(1e-2, max(eps_floor, safety * eps / res)): the relative
// reduction the next inner solve is asked for (at least 100x per round)
void launch_residual_check(int S, int nblk, const double* part, double eps, double eps_floor, double safety,
                           double* res, double* rnorm, int* outer, int* n_outer, double* eps_sys, cudaStream_t st);
// v32 = r64 / rn (per system) where outer; other systems inactive
template <typename Rl> void launch_make_inner_rhs(int S, int n3, const double2* r, const double* rnorm, const int* outer,
                                                  cx<Rl>* v, int* active, int* n_active, cudaStream_t st);
// x64 += rn * x_inner (systems with outer[s])
template <typename Rl> void launch_accumulate(int S, int n3, const cx<Rl>* xi, const double* rnorm, const int* outer,
                                              double2* x, cudaStream_t st);
// r = b - y
void launch_sub(int S, int n3, const double2* b, const double2* y, double2* r, cudaStream_t st);
// FP32 copy of an FP64 vector batch and back
void launch_to_f32(size_t n, const double2* a, float2* b, cudaStream_t st);

// ---- Loss reductions (Eq. 32, 17, 18) on u = coef * x (scaled dipoles) ----
// per system sums: [0..1] sum E_a . u, [2..3] sum conj(E_inc) . u, [4] sum |u|^2 w_abs[mat]
void launch_losses(const LatticeDev& L, int S, const double2* e, const double2* x, const double2* coef,
                   const double* wabs, const double* wdv, const SysField* sys, double* part, int nblk, double* sums,
                   cudaStream_t st);
// u = coef * x in FP32 and FP64
void launch_scaled_dipoles(const LatticeDev& L, int S, const double2* x, const double2* coef, double2* u64, float2* u32,
                           cudaStream_t st);
// Far field: sums[s] = sum_n w_n |F'(n)|^2, F'(n) = (I - nn) sum_j u_j exp(-i kappa n.r_j)
template <typename Rl>
void launch_farfield(const LatticeDev& L, int S, const cx<Rl>* u, const double2* kappa_sys, const double* dirs,
                     const double* weights, int n_dir, double* part, double* sums, cudaStream_t st);

}  // namespace eels
