// Host engine and C ABI of libeelsdda (see include/eelsdda.h).
//
// A solve runs, per batch of (energy, beam) systems (energy-major order):
//   1. per energy: host scalars omega, m_h, beta_h, gamma_h (Eq. 24), k = m_h k0,
//      polarizabilities (Clausius-Mossotti with radiative reaction);
//   2. D-hat: FFT of the Green's tensor (Eq. 5) on the padded lattice (FP64,
//      also rounded to FP32), one per energy, shared by that energy's beams;
//   3. incident field (Eq. 25) per (system, dipole), FP64;
//   4. the Jacobi-scaled system (I - a^1/2 G~ a^1/2) y = a^1/2 E is solved by
//      FP64 iterative refinement: r = b - A x in FP64, an inner QMR solve of
//      A d = r (FP32 in EELS_MIXED, FP64 in EELS_FP64), x += d, until
//      ||r|| <= eps_it ||b||;
//   5. loss sums (Eq. 32, 17, 18) in FP64 and the CL far field (Eq. 42).
// Lengths inside are in units of d and fields in units of the modulus of
// the Eq. 25 prefactor, so FP32 never meets the ~1e-37 magnitudes of SI
// dipole moments.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <mutex>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <limits>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/eelsdda.h"
#include "kernels.h"
#include "solve.h"

using cd = std::complex<double>;
using namespace eels;

namespace eels {
std::atomic<long long> g_kernel_launches{0};
thread_local bool g_capturing = false;
}  // namespace eels

namespace {

// Physical constants, SI (CODATA 2018; e, hbar, c exact).
constexpr double kE = 1.602176634e-19;
constexpr double kHbar = 1.054571817e-34;
constexpr double kC = 299792458.0;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kMeC2keV = 510.99895000;
constexpr double kPi = 3.14159265358979323846;

struct Fail {
    int code;
    std::string msg;
};

#define CK(call)                                                                                     \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess)                                                                       \
            throw Fail{e_ == cudaErrorMemoryAllocation ? EELS_E_OOM : EELS_E_CUDA,                   \
                       std::string(#call) + ": " + cudaGetErrorString(e_)};                          \
    } while (0)

// Device buffer that only grows; allocated stream-ordered on the owning
// context's stream, so one context's (re)allocation does not synchronise the
// device under other contexts' work.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    cudaStream_t* sp = nullptr;   // owning context's stream
    void ensure(size_t n) {
        if (n <= bytes) return;
        release();
        if (n == 0) return;
        cudaError_t e = sp ? cudaMallocAsync(&p, n, *sp) : cudaMalloc(&p, n);
        if (e != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            throw Fail{EELS_E_OOM, "device allocation of " + std::to_string(n) + " bytes failed"};
        }
        bytes = n;
    }
    void release() {
        if (p) {
            if (sp) cudaFreeAsync(p, *sp);
            else cudaFree(p);
        }
        p = nullptr;
        bytes = 0;
    }
    template <typename T> T* as() const { return reinterpret_cast<T*>(p); }
};

int good_fft_len(int n) {
    // smallest even 2^a 3^b 5^c 7^d >= 2n - 1 (any M >= 2n - 1 embeds the convolution)
    int m = std::max(2, 2 * n - 1);
    for (;; ++m) {
        if (m & 1) continue;
        int r = m;
        for (int p : {2, 3, 5, 7})
            while (r % p == 0) r /= p;
        if (r == 1) return m;
    }
}

// Padded length along x: 64 or 128 when that embeds the lattice (the
// register-resident x pass runs those lengths), else the smallest even
// 7-smooth length (any M >= 2n - 1 embeds the convolution).
int pad_len_x(int n) {
    const int need = 2 * n - 1;
    if (need > 32 && need <= 64) return 64;
    if (need > 64 && need <= 128) return 128;
    return good_fft_len(n);
}

FftPlan make_plan(int L) {
    FftPlan p{};
    p.L = L;
    int r = L;
    std::vector<int> rad;
    // power-of-two radices first (largest first: fewer passes over shared
    // memory, and Ns stays a power of two for shift/mask indexing), then 3, 5, 7
    while (r % 8 == 0) { rad.push_back(8); r /= 8; }
    while (r % 4 == 0) { rad.push_back(4); r /= 4; }
    while (r % 2 == 0) { rad.push_back(2); r /= 2; }
    for (int q : {3, 5, 7}) while (r % q == 0) { rad.push_back(q); r /= q; }
    auto log2_or_neg = [](int v) {
        if (v <= 0 || (v & (v - 1))) return -1;
        int s = 0;
        while ((1 << s) < v) ++s;
        return s;
    };
    p.nst = (int)rad.size();
    int Ns = 1;
    for (int i = 0; i < p.nst; ++i) {
        FftStage& sd = p.st[i];
        sd.R = rad[i];
        sd.Ns = Ns;
        sd.ns_shift = log2_or_neg(Ns);
        sd.nb = L / sd.R;
        sd.nb_shift = log2_or_neg(sd.nb);
        sd.ts = L / (Ns * sd.R);
        Ns *= sd.R;
    }
    return p;
}

// Icosphere: level-L subdivided icosahedron, vertex weights = 1/3 of the
// adjacent spherical-triangle areas (sum 4 pi).
bool icosphere(int n_dir, std::vector<double>& dirs, std::vector<double>& wts) {
    int level = -1;
    for (int l = 0; l <= 7; ++l)
        if (10 * (1 << (2 * l)) + 2 == n_dir) level = l;
    if (level < 0) return false;
    const double t = (1.0 + std::sqrt(5.0)) / 2.0;
    std::vector<std::array<double, 3>> V = {{-1, t, 0}, {1, t, 0}, {-1, -t, 0}, {1, -t, 0}, {0, -1, t}, {0, 1, t},
                                            {0, -1, -t}, {0, 1, -t}, {t, 0, -1}, {t, 0, 1}, {-t, 0, -1}, {-t, 0, 1}};
    for (auto& v : V) {
        double n = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        for (auto& c : v) c /= n;
    }
    std::vector<std::array<int, 3>> F = {{0, 11, 5}, {0, 5, 1}, {0, 1, 7}, {0, 7, 10}, {0, 10, 11}, {1, 5, 9}, {5, 11, 4},
                                         {11, 10, 2}, {10, 7, 6}, {7, 1, 8}, {3, 9, 4}, {3, 4, 2}, {3, 2, 6}, {3, 6, 8},
                                         {3, 8, 9}, {4, 9, 5}, {2, 4, 11}, {6, 2, 10}, {8, 6, 7}, {9, 8, 1}};
    for (int l = 0; l < level; ++l) {
        std::map<std::pair<int, int>, int> cache;
        auto mid = [&](int a, int b) {
            auto key = std::make_pair(std::min(a, b), std::max(a, b));
            auto it = cache.find(key);
            if (it != cache.end()) return it->second;
            std::array<double, 3> m;
            for (int c = 0; c < 3; ++c) m[c] = V[a][c] + V[b][c];
            double n = std::sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
            for (auto& c : m) c /= n;
            V.push_back(m);
            cache[key] = (int)V.size() - 1;
            return (int)V.size() - 1;
        };
        std::vector<std::array<int, 3>> nf;
        for (auto& f : F) {
            int ab = mid(f[0], f[1]), bc = mid(f[1], f[2]), ca = mid(f[2], f[0]);
            nf.push_back({f[0], ab, ca});
            nf.push_back({f[1], bc, ab});
            nf.push_back({f[2], ca, bc});
            nf.push_back({ab, bc, ca});
        }
        F.swap(nf);
    }
    dirs.assign(3 * V.size(), 0.0);
    wts.assign(V.size(), 0.0);
    for (size_t i = 0; i < V.size(); ++i)
        for (int c = 0; c < 3; ++c) dirs[3 * i + c] = V[i][c];
    for (auto& f : F) {
        const auto &a = V[f[0]], &b = V[f[1]], &c = V[f[2]];
        // solid angle of the spherical triangle (Van Oosterom & Strackee)
        double bxc[3] = {b[1] * c[2] - b[2] * c[1], b[2] * c[0] - b[0] * c[2], b[0] * c[1] - b[1] * c[0]};
        double num = std::fabs(a[0] * bxc[0] + a[1] * bxc[1] + a[2] * bxc[2]);
        double ab = a[0] * b[0] + a[1] * b[1] + a[2] * b[2], bc = b[0] * c[0] + b[1] * c[1] + b[2] * c[2],
               ca = c[0] * a[0] + c[1] * a[1] + c[2] * a[2];
        double om = 2.0 * std::atan2(num, 1.0 + ab + bc + ca);
        for (int k = 0; k < 3; ++k) wts[f[k]] += om / 3.0;
    }
    return true;
}

double2 d2(cd z) { return make_double2(z.real(), z.imag()); }
cd cz(eels_c128 z) { return cd(z.re, z.im); }

// Per-energy scalars.
struct EnergyPar {
    double omega;
    cd eps_h, m_h, beta, gamma, k, kappa;
    double scale;        // |q w / (2 pi eps0 m_h^2 v^2 gamma_h)|
    cd pref_unit;
    double wdv;
    cd alpha[EELS_MAX_MAT], sa[EELS_MAX_MAT], alpha_inv[EELS_MAX_MAT];
    double wabs[EELS_MAX_MAT];   // -Im 1/alpha'_CM
};

}  // namespace

struct eels_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    // lattice
    bool has_grid = false;
    int nx = 0, ny = 0, nz = 0, N = 0;
    double d_nm = 0;
    double origin[3] = {0, 0, 0};  // lattice centre in the frame of the beams (lattice units)
    std::vector<int> cellmap_h;    // ABI layout cell -> ABI dipole index (x-fastest order), -1 empty
    std::vector<int> dip_cell_h;   // internal dipole -> cell index
    std::vector<int> abi_of;       // internal dipole -> ABI dipole index
    std::vector<uint8_t> mat_h;    // internal dipole -> material (0-based)
    int max_mat = 0;
    LatticeDev L{};
    DevBuf cellmap, mat, dip_cell, col_range, colinfo, tw64[3], tw32[3];
    // workspace
    DevBuf e64, b64, x64, r64, y64, U, u64, u32;
    DevBuf kv[7];                                          // Krylov vectors V0 V1 P0 P1 P2 W X
    DevBuf part_a, part_b, qmr, bicg, active, upd, counters, outer, res, rnorm, eps_sys;
    DevBuf sysf, coef, diag, wabs, wdv, slot, kappa_sys;
    DevBuf G, Dr64, Dr32, Dx32, kappa_slot, igt_tab;
    int interaction = EELS_INT_POINT, polarizability = EELS_POL_CM;   // eels_set_interaction
    DevBuf lpart, lsums, fpart, fsums, dirs, wts;
    int dirs_n = 0;
    int* pinned = nullptr;
    // cached inner-loop graph
    cudaGraphExec_t graph = nullptr;
    bool tuned = false;            // x-pass tile widths timed for the current lattice
    std::vector<const void*> graph_key;
    long long graph_kernels = 0;
    // operator prepared by eels_prepare_operator
    int op_systems = 0;
    // consecutive systems that share a D-hat slot (the beams of one energy):
    // the x pass reuses a staged D-hat tile over up to this many of them;
    // spb_tuned is the autotuner's choice for the lattice (0: not tuned yet)
    int spb = 1, spb_tuned = 0;
    // the autotuner's choices per lattice shape (dims, padded dims, column
    // structure, materials), kept across eels_set_grid calls
    struct Tuned { int xw32, xw64, xmode, spb; std::vector<std::array<float, 3>> log; };
    std::vector<std::array<float, 3>> xreg_log;   // the register x pass's timed candidates
    std::map<std::array<int, 8>, Tuned> tune_cache;
    std::array<int, 8> shape_key() const {
        return {L.Nx, L.Ny, L.Nz, L.Mx, L.My, L.Mz, L.contig, L.nmat};
    }

    std::vector<DevBuf*> buffers() {
        std::vector<DevBuf*> v = {&cellmap, &mat, &dip_cell, &col_range, &colinfo, &e64, &b64, &x64, &r64, &y64, &U, &u64, &u32,
                                  &part_a, &part_b, &qmr, &bicg, &active, &upd, &counters, &outer, &res, &rnorm, &eps_sys,
                                  &sysf, &coef, &diag, &wabs, &wdv, &slot, &kappa_sys, &G, &Dr64, &Dr32, &Dx32, &kappa_slot, &igt_tab,
                                  &lpart, &lsums, &fpart, &fsums, &dirs, &wts};
        for (auto& b : kv) v.push_back(&b);
        for (auto& b : tw64) v.push_back(&b);
        for (auto& b : tw32) v.push_back(&b);
        return v;
    }
};

namespace {

void set_err(eels_ctx* c, const std::string& m) {
    if (c) c->err = m;
}

template <typename T> void h2d(DevBuf& b, const std::vector<T>& v, cudaStream_t st) {
    b.ensure(std::max<size_t>(v.size() * sizeof(T), 16));
    if (!v.empty()) CK(cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
}

void upload_twiddles(eels_ctx* c, int axis, int M) {
    std::vector<double2> t64(M);
    std::vector<float2> t32(M);
    for (int t = 0; t < M; ++t) {
        // exp(-2 pi i t / M), argument reduced exactly in long double
        long double a = -2.0L * 3.14159265358979323846264338327950288L * (long double)t / (long double)M;
        double cr = (double)std::cos(a), ci = (double)std::sin(a);
        t64[t] = make_double2(cr, ci);
        t32[t] = make_float2((float)cr, (float)ci);
    }
    h2d(c->tw64[axis], t64, c->stream);
    h2d(c->tw32[axis], t32, c->stream);
}

void set_grid(eels_ctx* c, const eels_grid* g) {
    if (!g || g->nx <= 0 || g->ny <= 0 || g->nz <= 0 || !(g->d_nm > 0) || !g->occ)
        throw Fail{EELS_E_INVALID_ARG, "grid: extents and d must be positive and occ non-NULL"};
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(g->origin_nm[a])) throw Fail{EELS_E_INVALID_ARG, "grid: origin must be finite"};
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    const size_t ncell = (size_t)nx * ny * nz;
    // ABI numbering: occupied cells in x-fastest order (cellmap_h: cell -> ABI index)
    c->cellmap_h.assign(ncell, -1);
    int maxm = 0, nabi = 0;
    for (size_t i = 0; i < ncell; ++i) {
        const int m = g->occ[i];
        if (m == 0) continue;
        if (m > EELS_MAX_MAT) throw Fail{EELS_E_INVALID_ARG, "grid: material index > 8"};
        c->cellmap_h[i] = nabi++;
        maxm = std::max(maxm, m);
    }
    if (nabi == 0) throw Fail{EELS_E_INVALID_ARG, "grid: no occupied cell"};
    // internal numbering: slab-major (ix, iy, iz), z fastest, so that every
    // x-slab's dipoles are contiguous for the FFT slab kernels
    std::vector<int> cm_dev(ncell, -1);
    c->abi_of.clear();
    c->dip_cell_h.clear();
    c->mat_h.clear();
    for (int ix = 0; ix < nx; ++ix)
        for (int iy = 0; iy < ny; ++iy)
            for (int iz = 0; iz < nz; ++iz) {
                const size_t cell = (size_t)ix + (size_t)nx * (iy + (size_t)ny * iz);
                const int a = c->cellmap_h[cell];
                if (a < 0) continue;
                cm_dev[((size_t)ix * ny + iy) * nz + iz] = (int)c->abi_of.size();
                c->abi_of.push_back(a);
                c->dip_cell_h.push_back((int)cell);
                c->mat_h.push_back((uint8_t)(g->occ[cell] - 1));
            }
    const int Mx = pad_len_x(nx), My = good_fft_len(ny), Mz = good_fft_len(nz);
    if (Mx > 256 || My > 256 || Mz > 256)
        throw Fail{EELS_E_UNSUPPORTED, "grid: padded FFT length above 256 (extent above 128 cells)"};
    std::vector<int2> cr((size_t)nx * ny, make_int2(0, 0));
    for (int iy = 0; iy < ny; ++iy)
        for (int ix = 0; ix < nx; ++ix) {
            int first = -1, last = -1;
            for (int iz = 0; iz < nz; ++iz)
                if (c->cellmap_h[((size_t)iz * ny + iy) * nx + ix] >= 0) {
                    if (first < 0) first = iz;
                    last = iz;
                }
            if (first >= 0) cr[(size_t)iy * nx + ix] = make_int2(first, last + 1);
        }
    // per (ix, iy) column in the internal numbering: index of its first dipole
    // minus its first iz, the occupied iz range, and whether every column's
    // occupied cells are contiguous (then dipole = colinfo.x + iz exactly)
    std::vector<int4> ci((size_t)nx * ny, make_int4(0, 0, 0, 0));
    bool contig = true;
    {
        int next = 0;
        for (int ix = 0; ix < nx; ++ix)
            for (int iy = 0; iy < ny; ++iy) {
                const int2 r = cr[(size_t)iy * nx + ix];
                int cnt = 0;
                for (int iz = 0; iz < nz; ++iz) cnt += c->cellmap_h[((size_t)iz * ny + iy) * nx + ix] >= 0;
                if (cnt != r.y - r.x) contig = false;
                ci[(size_t)ix * ny + iy] = make_int4(next - r.x, r.x, r.y, 0);
                next += cnt;
            }
    }
    c->nx = nx; c->ny = ny; c->nz = nz;
    c->N = (int)c->dip_cell_h.size();
    c->d_nm = g->d_nm;
    for (int a = 0; a < 3; ++a) c->origin[a] = g->origin_nm[a] / g->d_nm;
    c->max_mat = maxm;
    CK(cudaSetDevice(c->device));
    h2d(c->cellmap, cm_dev, c->stream);
    h2d(c->mat, c->mat_h, c->stream);
    h2d(c->dip_cell, c->dip_cell_h, c->stream);
    h2d(c->col_range, cr, c->stream);
    h2d(c->colinfo, ci, c->stream);
    upload_twiddles(c, 0, Mx);
    upload_twiddles(c, 1, My);
    upload_twiddles(c, 2, Mz);
    LatticeDev& L = c->L;
    L.Nx = nx; L.Ny = ny; L.Nz = nz; L.N = c->N;
    L.Mx = Mx; L.My = My; L.Mz = Mz;
    L.Hx = Mx / 2 + 1; L.Hy = My / 2 + 1; L.Hz = Mz / 2 + 1;
    L.cellmap = c->cellmap.as<int>();
    L.mat = c->mat.as<uint8_t>();
    L.dip_cell = c->dip_cell.as<int>();
    L.col_range = c->col_range.as<int2>();
    L.colinfo = c->colinfo.as<int4>();
    L.contig = contig ? 1 : 0;
    L.nmat = maxm;
    L.px = make_plan(Mx); L.py = make_plan(My); L.pz = make_plan(Mz);
    L.tw64x = c->tw64[0].as<double2>(); L.tw64y = c->tw64[1].as<double2>(); L.tw64z = c->tw64[2].as<double2>();
    L.tw32x = c->tw32[0].as<float2>(); L.tw32y = c->tw32[1].as<float2>(); L.tw32z = c->tw32[2].as<float2>();
    if (matvec_smem_bytes(L, true) == 0) throw Fail{EELS_E_UNSUPPORTED, "grid: FFT tiles do not fit shared memory"};
    CK(cudaStreamSynchronize(c->stream));
    c->has_grid = true;
    c->tuned = false;
    c->L.xw32 = c->L.xw64 = 0;
    c->L.xmode = 0;
    c->spb_tuned = 0;
    const auto t = c->tune_cache.find(c->shape_key());
    if (t != c->tune_cache.end()) {
        c->L.xw32 = t->second.xw32;
        c->L.xw64 = t->second.xw64;
        c->L.xmode = t->second.xmode;
        c->spb_tuned = t->second.spb;
        c->xreg_log = t->second.log;
        c->tuned = true;
    } else {
        c->xreg_log.clear();
    }
    if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
}

double electron_speed(double ekin_keV) {
    const double g = 1.0 + ekin_keV / kMeC2keV;
    return kC * std::sqrt(1.0 - 1.0 / (g * g));
}

// pol: EELS_POL_CM (Clausius-Mossotti with radiative reaction) or
// EELS_POL_IGT_SO (the cell's self term to second order in kd, igt.cu).
EnergyPar energy_params(double ekin, double e_eV, cd eps_h, int n_mat, const eels_c128* eps_p, double d_m,
                        int pol = EELS_POL_CM) {
    if (!(e_eV > 0)) throw Fail{EELS_E_INVALID_ARG, "energies must be positive"};
    if (eps_h.imag() < 0) throw Fail{EELS_E_INVALID_ARG, "Im eps_h < 0: active host medium (excluded, Sec. 2.1)"};
    EnergyPar p{};
    const double v = electron_speed(ekin);
    p.omega = e_eV * kE / kHbar;
    p.eps_h = eps_h;
    p.m_h = std::sqrt(eps_h);                 // principal branch
    p.beta = v / kC * p.m_h;
    const cd a = 1.0 - p.beta * p.beta;
    if (std::abs(a) < 1e-12) throw Fail{EELS_E_THRESHOLD, "|1 - beta_h^2| < 1e-12: gamma_h singular (Eq. 24)"};
    cd s = (a.imag() == 0.0 && a.real() < 0.0) ? cd(0.0, -std::sqrt(-a.real())) : std::sqrt(a);   // 1/gamma_h
    p.gamma = 1.0 / s;
    p.k = p.m_h * p.omega / kC;
    p.kappa = p.k * d_m;
    const cd pref = -kE * p.omega / (2.0 * kPi * kEps0 * p.m_h * p.m_h * v * v * p.gamma);
    p.scale = std::abs(pref);
    p.pref_unit = pref / p.scale;
    p.wdv = p.omega * d_m / v;
    const cd k3 = p.kappa * p.kappa * p.kappa;
    for (int m = 0; m < n_mat; ++m) {
        const cd m2 = cz(eps_p[m]) / eps_h;                                     // m^2 = eps_p / eps_h
        const cd acm = 3.0 / (4.0 * kPi) * (m2 - 1.0) / (m2 + 2.0);           // alpha'_CM = alpha~_CM / d^3
        // 1/alpha' = 1/alpha'_CM - (2/3) i kappa^3 (radiative reaction), and
        // with igt_so also - (2/3) c1 kappa^2 (the k^2 term of the cell's self field)
        cd self = cd(0.0, 2.0 / 3.0) * k3;
        if (pol == EELS_POL_IGT_SO) self += (2.0 / 3.0) * IGT_C1 * p.kappa * p.kappa;
        const cd al = acm / (1.0 - self * acm);
        p.alpha[m] = al;
        p.sa[m] = std::sqrt(al);
        p.alpha_inv[m] = 1.0 / al;
        p.wabs[m] = -(1.0 / acm).imag();
    }
    return p;
}

// Frame (e1, e2, n) of an electron moving along dir: the smallest rotation
// taking z to n applied to (x, y, z) (Rodrigues' formula about z x n; a half
// turn about x when n = -z).  The trajectory passes through x0 e1 + y0 e2.
struct BeamFrame {
    double e1[3], e2[3], n[3];
    bool along_z;
};

BeamFrame beam_frame(const double* dir) {
    BeamFrame f{};
    const double len = std::sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
    if (!(len > 0) || !std::isfinite(len)) throw Fail{EELS_E_INVALID_ARG, "beam_dir must be a finite non-zero vector"};
    const double n[3] = {dir[0] / len, dir[1] / len, dir[2] / len};
    double R[3][3];
    const double kx = -n[1], ky = n[0];                 // z x n
    const double sn = std::sqrt(kx * kx + ky * ky), cs = n[2];
    if (sn < 1e-15) {
        const double sg = cs > 0 ? 1.0 : -1.0;
        const double Rm[3][3] = {{1, 0, 0}, {0, sg, 0}, {0, 0, sg}};
        std::memcpy(R, Rm, sizeof(R));
    } else {
        const double ux = kx / sn, uy = ky / sn;      // unit axis (ux, uy, 0)
        const double K[3][3] = {{0, 0, uy}, {0, 0, -ux}, {-uy, ux, 0}};
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double kk = 0;
                for (int m = 0; m < 3; ++m) kk += K[i][m] * K[m][j];
                R[i][j] = (i == j ? 1.0 : 0.0) + sn * K[i][j] + (1.0 - cs) * kk;
            }
    }
    for (int i = 0; i < 3; ++i) {
        f.e1[i] = R[i][0];
        f.e2[i] = R[i][1];
        f.n[i] = R[i][2];
    }
    f.along_z = dir[0] == 0.0 && dir[1] == 0.0 && dir[2] > 0.0;
    if (f.along_z) {
        const double e1[3] = {1, 0, 0}, e2[3] = {0, 1, 0}, ez[3] = {0, 0, 1};
        std::memcpy(f.e1, e1, sizeof(e1));
        std::memcpy(f.e2, e2, sizeof(e2));
        std::memcpy(f.n, ez, sizeof(ez));
    }
    return f;
}

// The z-electron kernels take the phase at z = 0 of the lattice frame: they
// apply while the lattice centre has no z offset in the frame of the beams.
bool z_path(const eels_ctx* c, const BeamFrame& f) { return f.along_z && c->origin[2] == 0.0; }

// Fills the electron fields of a SysField for beam b in lattice units,
// relative to the lattice centre: the trajectory through x0 e1 + y0 e2 of the
// beams' frame, where the lattice centre sits at `origin`.
void set_beam(SysField& sf, const BeamFrame& f, const eels_beam& beam, const eels_ctx* c) {
    const double x0 = beam.x0_nm / c->d_nm, y0 = beam.y0_nm / c->d_nm;
    sf.x0 = x0 - c->origin[0];
    sf.y0 = y0 - c->origin[1];
    sf.px = x0 * f.e1[0] + y0 * f.e2[0] - c->origin[0];
    sf.py = x0 * f.e1[1] + y0 * f.e2[1] - c->origin[1];
    sf.pz = x0 * f.e1[2] + y0 * f.e2[2] - c->origin[2];
    sf.nx = f.n[0];
    sf.ny = f.n[1];
    sf.nz = f.n[2];
    sf.along_z = z_path(c, f) ? 1 : 0;
}

// An oblique electron must not cross an occupied cell: slab test of the line
// p + t n against every occupied unit cube (lattice units).
void check_beams_dir(eels_ctx* c, int n_beam, const eels_beam* beams, const BeamFrame& f) {
    for (int b = 0; b < n_beam; ++b) {
        SysField sf{};
        set_beam(sf, f, beams[b], c);
        const double p[3] = {sf.px, sf.py, sf.pz}, n[3] = {f.n[0], f.n[1], f.n[2]};
        if (!std::isfinite(p[0]) || !std::isfinite(p[1]) || !std::isfinite(p[2]))
            throw Fail{EELS_E_INVALID_ARG, "beam position not finite"};
        for (int iz = 0; iz < c->nz; ++iz)
            for (int iy = 0; iy < c->ny; ++iy)
                for (int ix = 0; ix < c->nx; ++ix) {
                    if (c->cellmap_h[((size_t)iz * c->ny + iy) * c->nx + ix] < 0) continue;
                    const double lo[3] = {ix - 0.5 * c->nx, iy - 0.5 * c->ny, iz - 0.5 * c->nz};
                    double t0 = -1e300, t1 = 1e300;
                    bool hit = true;
                    for (int a = 0; a < 3 && hit; ++a) {
                        if (std::fabs(n[a]) < 1e-300) {
                            hit = p[a] >= lo[a] && p[a] <= lo[a] + 1.0;
                        } else {
                            double ta = (lo[a] - p[a]) / n[a], tb = (lo[a] + 1.0 - p[a]) / n[a];
                            if (ta > tb) std::swap(ta, tb);
                            t0 = std::max(t0, ta);
                            t1 = std::min(t1, tb);
                            hit = t0 <= t1;
                        }
                    }
                    if (hit) throw Fail{EELS_E_BEAM_INSIDE, "beam " + std::to_string(b) + " crosses an occupied cell"};
                }
    }
}

void check_beams(eels_ctx* c, int n_beam, const eels_beam* beams) {
    for (int b = 0; b < n_beam; ++b) {
        const double x = beams[b].x0_nm / c->d_nm - c->origin[0] + 0.5 * c->nx,
                     y = beams[b].y0_nm / c->d_nm - c->origin[1] + 0.5 * c->ny;
        if (!std::isfinite(x) || !std::isfinite(y)) throw Fail{EELS_E_INVALID_ARG, "beam position not finite"};
        const int ix = (int)std::floor(x), iy = (int)std::floor(y);
        // the line crosses a cell (or touches its boundary) whose column holds a dipole
        for (int jx = ix - 1; jx <= ix + 1; ++jx)
            for (int jy = iy - 1; jy <= iy + 1; ++jy) {
                if (jx < 0 || jy < 0 || jx >= c->nx || jy >= c->ny) continue;
                if (x < jx || x > jx + 1 || y < jy || y > jy + 1) continue;
                for (int iz = 0; iz < c->nz; ++iz)
                    if (c->cellmap_h[((size_t)iz * c->ny + jy) * c->nx + jx] >= 0)
                        throw Fail{EELS_E_BEAM_INSIDE, "beam " + std::to_string(b) + " crosses an occupied cell"};
            }
    }
}

size_t per_system_bytes(const LatticeDev& L, bool fp64) {
    const size_t n3 = (size_t)3 * L.N;
    const size_t vec64 = n3 * sizeof(double2);
    const size_t kvec = n3 * (fp64 ? sizeof(double2) : sizeof(float2));
    const size_t u = (size_t)3 * L.My * L.Nx * L.Mz * sizeof(double2);
    const int nblk = (int)((n3 + RED_CHUNK - 1) / RED_CHUNK);
    return 6 * vec64 + n3 * sizeof(float2) + u + 7 * kvec + 2 * (size_t)nblk * 4 * sizeof(double) + 1024;
}

size_t per_slot_bytes(const LatticeDev& L) {
    return (size_t)6 * L.Hx * L.Hy * L.Hz * (sizeof(double2) + 2 * sizeof(float2));
}

// The lattice description for a D-hat build with the given interaction term
// (uploads the igt_so cell tables on first use).
LatticeDev dhat_lattice(eels_ctx* c, int interaction) {
    LatticeDev L = c->L;
    L.igt = nullptr;
    if (interaction == EELS_INT_IGT_SO) {
        if (!c->igt_tab.p) h2d(c->igt_tab, igt_tables(), c->stream);
        L.igt = c->igt_tab.as<double>();
    }
    return L;
}

// Iterations allowed per inner solve: an FP32 inner solve may be restarted
// early (inner_max_iter) so that rounding in FP32 does not let it stagnate.
int inner_cap(const eels_opts* o, bool fp32) {
    return (fp32 && o->inner_max_iter > 0) ? std::min(o->max_iter, o->inner_max_iter) : o->max_iter;
}

struct Batch {
    int S, e0, e1;   // systems, first/last+1 energy
};

// ------------------------------------------------------------------ solve
template <typename Rl>
KrylovArgs<Rl> krylov_args(eels_ctx* c, int S, const eels_opts* o, double eps) {
    KrylovArgs<Rl> k{};
    const int n3 = 3 * c->N;
    k.S = S;
    k.n3 = n3;
    k.nblk = (n3 + RED_CHUNK - 1) / RED_CHUNK;
    k.nblk_a = k.nblk;
    k.V[0] = c->kv[0].as<cx<Rl>>(); k.V[1] = c->kv[1].as<cx<Rl>>();
    k.P[0] = c->kv[2].as<cx<Rl>>(); k.P[1] = c->kv[3].as<cx<Rl>>(); k.P[2] = c->kv[4].as<cx<Rl>>();
    k.W = c->kv[5].as<cx<Rl>>(); k.X = c->kv[6].as<cx<Rl>>();
    k.part_a = c->part_a.as<double>(); k.part_b = c->part_b.as<double>();
    k.qmr = c->qmr.as<QmrState>();
    k.qmr2 = c->qmr.as<Qmr2State>();
    // BiCGStab roles in the same seven buffers (the rhs arrives in kv[1], the iterate is kv[6])
    k.R = c->kv[1].as<cx<Rl>>(); k.Rh = c->kv[0].as<cx<Rl>>(); k.Pb = c->kv[2].as<cx<Rl>>();
    k.Vb = c->kv[3].as<cx<Rl>>(); k.Tb = c->kv[4].as<cx<Rl>>(); k.Sb = k.R;
    k.bicg = c->bicg.as<BicgState>();
    k.active = c->active.as<int>(); k.upd = c->upd.as<int>();
    k.n_active = c->counters.as<int>();
    k.eps = eps;
    k.eps_sys = c->eps_sys.as<double>();
    k.max_iter = inner_cap(o, sizeof(Rl) == 4);
    return k;
}

template <typename Rl>
MatvecArgs<Rl> mv_args(eels_ctx* c, int S, const cx<Rl>* x, cx<Rl>* y, const cx<Rl>* Dr, const int* active, bool scaled) {
    MatvecArgs<Rl> a{};
    a.x = x; a.y = y; a.U = c->U.as<cx<Rl>>(); a.Dr = Dr;
    a.sys_slot = c->slot.as<int>();
    a.coef = c->coef.as<double2>();
    a.diag = c->diag.as<double2>();
    a.active = active;
    a.Dx = sizeof(Rl) == 4 ? c->Dx32.as<float2>() : nullptr;
    a.S = S;
    a.spb = c->spb;
    (void)scaled;
    return a;
}

template <typename Rl> const cx<Rl>* dr_of(eels_ctx* c);
template <> const float2* dr_of<float>(eels_ctx* c) { return c->Dr32.as<float2>(); }
template <> const double2* dr_of<double>(eels_ctx* c) { return c->Dr64.as<double2>(); }

// Inner Krylov solve (QMR or BiCGStab) on the active systems; returns the
// number of iterations run.
template <typename Rl>
int inner_solve(eels_ctx* c, int S, const eels_opts* o, double eps) {
    cudaStream_t st = c->stream;
    KrylovArgs<Rl> k = krylov_args<Rl>(c, S, o, eps);
    const bool bicg = o->solver == EELS_BICGSTAB, qmr2 = o->solver == EELS_QMR2;
    // the three-pass matvec also returns the per-slab partial sums of x^T (A x)
    const bool fused = !bicg && matvec_passes(c->L, sizeof(Rl) == 8) == 3;
    k.nblk_a = fused ? 3 * c->L.Nx : k.nblk;
    if (bicg) launch_bicg_init<Rl>(k, st);
    else if (qmr2) launch_qmr2_init<Rl>(k, st);
    else launch_qmr_init<Rl>(k, st);
    CK(cudaGetLastError());
    constexpr int CHUNK = 6;   // period of the QMR vector-slot rotation (2 and 3)
    // every pointer and scalar baked into the captured kernels
    std::vector<const void*> key = {k.V[0], k.V[1], k.P[0], k.P[1], k.P[2], k.W, k.X, c->U.p, dr_of<Rl>(c),
                                    (const void*)(size_t)S, (const void*)(size_t)sizeof(Rl),
                                    (const void*)(size_t)inner_cap(o, sizeof(Rl) == 4), c->coef.p, c->diag.p, c->slot.p, c->qmr.p,
                                    c->part_a.p, c->part_b.p, c->active.p, c->upd.p, c->counters.p, c->eps_sys.p,
                                    c->cellmap.p, c->bicg.p, (const void*)(size_t)o->solver,
                                    (const void*)(size_t)c->spb, c->Dx32.p};
    // eps is read inside the step kernel from the kernel argument: make it part of the key
    double epsv = eps;
    const void* ek;
    std::memcpy(&ek, &epsv, sizeof(ek));
    key.push_back(ek);
    const bool dev_loop = o->device_loop != 0;
    key.push_back((const void*)(size_t)dev_loop);
    const int max_chunks = inner_cap(o, sizeof(Rl) == 4) / CHUNK + 2;
    int* chunks = c->counters.as<int>() + 2;
    if (!c->graph || c->graph_key != key) {
        if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
        // The graph holds CHUNK captured iterations.  With the device loop it
        // is a WHILE node whose body runs them and then the loop-control
        // kernel, which ends the loop once no system is active or max_chunks
        // chunks have run; without, the captured iterations are the graph.
        cudaGraph_t g;
        CK(cudaGraphCreate(&g, 0));
        struct GraphGuard { cudaGraph_t g; ~GraphGuard() { cudaGraphDestroy(g); } } gguard{g};
        cudaGraph_t body = g;
        cudaGraphConditionalHandle cond{};
        if (dev_loop) {
            CK(cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault));
            cudaGraphNodeParams np{};
            np.type = cudaGraphNodeTypeConditional;
            np.conditional.handle = cond;
            np.conditional.type = cudaGraphCondTypeWhile;
            np.conditional.size = 1;
            cudaGraphNode_t cnode;
            CK(cudaGraphAddNode(&cnode, g, nullptr, nullptr, 0, &np));
            body = np.conditional.phGraph_out[0];
        }
        CK(cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        g_capturing = true;
        // a launch that fails inside the capture throws: end the capture on the way out
        struct CaptureGuard {
            cudaStream_t st;
            ~CaptureGuard() {
                if (!g_capturing) return;
                g_capturing = false;
                cudaGraph_t partial = nullptr;
                cudaStreamEndCapture(st, &partial);
                cudaGetLastError();
            }
        } cguard{st};
        for (int n = 1; n <= CHUNK; ++n) {
            if (bicg) {
                launch_matvec<Rl>(c->L, mv_args<Rl>(c, S, k.Pb, k.Vb, dr_of<Rl>(c), k.active, true), st);
                launch_bicg_stage1<Rl>(k, st);
                launch_matvec<Rl>(c->L, mv_args<Rl>(c, S, k.R, k.Tb, dr_of<Rl>(c), k.active, true), st);
                launch_bicg_stage2<Rl>(k, st);
                continue;
            }
            if (qmr2) {
                MatvecArgs<Rl> a = mv_args<Rl>(c, S, k.P[0], k.W, dr_of<Rl>(c), k.active, true);
                a.dot_part = fused ? k.part_a : nullptr;
                launch_matvec<Rl>(c->L, a, st);
                launch_qmr2_post_matvec<Rl>(k, fused, st);
                continue;
            }
            MatvecArgs<Rl> a = mv_args<Rl>(c, S, k.V[n & 1], k.W, dr_of<Rl>(c), k.active, true);
            a.dot_part = fused ? k.part_a : nullptr;
            launch_matvec<Rl>(c->L, a, st);
            launch_qmr_post_matvec<Rl>(k, n, fused, st);
        }
        if (dev_loop) launch_loop_ctl(cond, k.n_active, chunks, max_chunks, st);
        g_capturing = false;
        cudaGraph_t captured;
        CK(cudaStreamEndCapture(st, &captured));
        CK(cudaGraphInstantiate(&c->graph, g, 0));
        // kernels per pass of the body (one chunk)
        size_t nn = 0;
        cudaGraphGetNodes(body, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        cudaGraphGetNodes(body, nodes.data(), &nn);
        c->graph_kernels = 0;
        for (auto& nd : nodes) {
            cudaGraphNodeType ty;
            cudaGraphNodeGetType(nd, &ty);
            if (ty == cudaGraphNodeTypeKernel) ++c->graph_kernels;
        }
        c->graph_key = key;
    }
    CK(cudaMemcpyAsync(c->pinned, k.n_active, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (*c->pinned <= 0) return 0;
    if (dev_loop) {
        // one launch per inner solve; the host waits once, for the chunk count
        CK(cudaMemsetAsync(chunks, 0, sizeof(int), st));
        CK(cudaGraphLaunch(c->graph, st));
        CK(cudaMemcpyAsync(c->pinned, chunks, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        const int n_chunks = *c->pinned;
        g_kernel_launches += (long long)n_chunks * c->graph_kernels;
        return n_chunks * CHUNK;
    }
    // The host reads the number of active systems between bursts of graph
    // replays; a burst grows from 1 to 8 replays as the solve goes on (a
    // replay after every system has converged only launches empty blocks).
    int it = 0, burst = 1;
    for (int ch = 0; ch < max_chunks;) {
        for (int b = 0; b < burst && ch < max_chunks; ++b, ++ch) {
            CK(cudaGraphLaunch(c->graph, st));
            g_kernel_launches += c->graph_kernels;
            it += CHUNK;
        }
        burst = std::min(8, burst * 2);
        CK(cudaMemcpyAsync(c->pinned, k.n_active, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (*c->pinned <= 0) break;
    }
    return it;
}

// Up to max_rounds refinement rounds with inner solves in precision Rl, on
// the systems whose FP64 residual is still above eps_it.  Returns how many
// systems are still above it after the last residual check.
template <typename Rl>
int refine_rounds(eels_ctx* c, int S, const eels_opts* o, int max_rounds, std::vector<int>& iters,
                  std::vector<int>& refin) {
    cudaStream_t st = c->stream;
    const int n3 = 3 * c->N;
    const int nblk = (n3 + RED_CHUNK - 1) / RED_CHUNK;
    int* n_outer = c->counters.as<int>() + 1;
    // inner tolerance per system: an FP32 solve is asked for eps_inner (or
    // what the next round still needs, if that is less demanding); an FP64
    // solve is asked for 0.5 eps_it / res, the reduction that reaches eps_it
    const double eps_floor = (sizeof(Rl) == 4) ? std::max(o->eps_inner, 1e-7) : 1e-15;
    const double safety = (sizeof(Rl) == 4) ? 0.3 : 0.5;
    std::vector<QmrState> qh(S);
    std::vector<Qmr2State> q2h(S);
    std::vector<BicgState> bh(S);
    std::vector<int> outer_h(S), slow_rounds(S, 0), stalled(S, 0);
    std::vector<double> res_h(S, 1.0), res_prev(S, 1.0);
    int left = 0;
    for (int round = 0; round <= max_rounds; ++round) {
        launch_norms2(S, n3, nblk, c->r64.as<double2>(), c->b64.as<double2>(), c->part_a.as<double>(), st);
        launch_residual_check(S, nblk, c->part_a.as<double>(), o->eps_it, eps_floor, safety, c->res.as<double>(),
                              c->rnorm.as<double>(), c->outer.as<int>(), n_outer, c->eps_sys.as<double>(), st);
        CK(cudaMemcpyAsync(c->pinned, n_outer, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        left = *c->pinned;
        if (left == 0 || round == max_rounds) break;
        if (sizeof(Rl) == 4) {
            // FP32 rounding can stall an inner solve: a system whose FP64
            // residual fell by less than 2x in each of the last two rounds
            // leaves the FP32 rounds (the FP64 rounds that follow take it);
            // the other systems go on in FP32
            CK(cudaMemcpyAsync(res_h.data(), c->res.p, S * sizeof(double), cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(outer_h.data(), c->outer.p, S * sizeof(int), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            int running = 0;
            bool masked = false;
            for (int s = 0; s < S; ++s) {
                const bool slow = outer_h[s] && round > 0 && res_h[s] > 0.5 * res_prev[s];
                slow_rounds[s] = slow ? slow_rounds[s] + 1 : 0;
                if (slow_rounds[s] >= 2) stalled[s] = 1;
                if (stalled[s] && outer_h[s]) {
                    outer_h[s] = 0;
                    masked = true;
                }
                running += outer_h[s];
                res_prev[s] = res_h[s];
            }
            if (running == 0) break;
            if (masked) CK(cudaMemcpyAsync(c->outer.p, outer_h.data(), S * sizeof(int), cudaMemcpyHostToDevice, st));
        }
        launch_make_inner_rhs<Rl>(S, n3, c->r64.as<double2>(), c->rnorm.as<double>(), c->outer.as<int>(),
                                  c->kv[1].as<cx<Rl>>(), c->active.as<int>(), c->counters.as<int>(), st);
        inner_solve<Rl>(c, S, o, eps_floor);
        if (o->solver == EELS_BICGSTAB) {
            CK(cudaMemcpyAsync(bh.data(), c->bicg.p, S * sizeof(BicgState), cudaMemcpyDeviceToHost, st));
        } else if (o->solver == EELS_QMR2) {
            CK(cudaMemcpyAsync(q2h.data(), c->qmr.p, S * sizeof(Qmr2State), cudaMemcpyDeviceToHost, st));
        } else {
            CK(cudaMemcpyAsync(qh.data(), c->qmr.p, S * sizeof(QmrState), cudaMemcpyDeviceToHost, st));
        }
        CK(cudaMemcpyAsync(outer_h.data(), c->outer.p, S * sizeof(int), cudaMemcpyDeviceToHost, st));
        launch_accumulate<Rl>(S, n3, c->kv[6].as<cx<Rl>>(), c->rnorm.as<double>(), c->outer.as<int>(),
                              c->x64.as<double2>(), st);
        // new residuals of the systems that took this round; the others keep
        // x, and y = A x from the round that last changed them
        MatvecArgs<double> a = mv_args<double>(c, S, c->x64.as<double2>(), c->y64.as<double2>(), c->Dr64.as<double2>(),
                                               c->outer.as<int>(), true);
        launch_matvec<double>(c->L, a, st);
        launch_sub(S, n3, c->b64.as<double2>(), c->y64.as<double2>(), c->r64.as<double2>(), st);
        CK(cudaStreamSynchronize(st));
        for (int s = 0; s < S; ++s)
            if (outer_h[s]) {
                iters[s] += o->solver == EELS_BICGSTAB ? bh[s].iters
                                                       : o->solver == EELS_QMR2 ? q2h[s].iters : qh[s].iters;
                refin[s] += 1;
            }
    }
    return left;
}

// FP64 refinement of a batch.  EELS_MIXED: FP32 inner solves restarted
// every inner_max_iter iterations.  With two-term QMR, up to 30 rounds; a
// system whose residual falls by less than 2x in two successive rounds
// leaves them for FP32 BiCGStab rounds (the complex-symmetric Lanczos process
// can stall or break down on a residual whose unconjugated square r^T r is
// small, where BiCGStab, with its conjugated inner product, does not).  With
// three-term QMR, whose FP32 recurrences lose biorthogonality much sooner,
// only two QMR rounds (most systems of a spectrum converge in them), then
// every system left goes to FP32 BiCGStab (on the 200-energy spectrum:
// 1.85 s per step against 2.49 s with 30 three-term QMR rounds).
// Systems still above eps_it finish with FP64 inner solves (BiCGStab after
// FP32 rounds, for the same reason).  Lattices whose padded FFT grid has at
// most 65,536 points (40^3) go straight to FP64 inner solves with the chosen
// solver: their matvec is bound by launch latency, so an FP64 iteration costs
// little more than an FP32 one, while restarted FP32 rounds need up to 3x
// the iterations on hard systems (measured on the serving stream: its rods
// and spheres up to 40^3 solve 2-7x faster in FP64, one 36^3 request 2x
// slower).  EELS_FP64: FP64 inner solves with the chosen solver.
void refine_batch(eels_ctx* c, int S, const eels_opts* o, bool fp64, std::vector<int>& iters, std::vector<int>& refin,
                  std::vector<double>& resid) {
    cudaStream_t st = c->stream;
    int left = 1;
    const size_t m_pad = (size_t)c->L.Mx * c->L.My * c->L.Mz;
    const bool fp32_rounds = !fp64 && m_pad > (size_t)65536;
    eels_opts ob = *o;
    ob.solver = EELS_BICGSTAB;
    if (fp32_rounds) {
        left = refine_rounds<float>(c, S, o, o->solver == EELS_QMR ? 2 : 30, iters, refin);
        if (left > 0 && o->solver != EELS_BICGSTAB) left = refine_rounds<float>(c, S, &ob, 30, iters, refin);
    }
    if (left > 0) {
        const size_t kvec64 = (size_t)S * 3 * c->N * sizeof(double2);
        for (auto& b : c->kv) b.ensure(kvec64);
        refine_rounds<double>(c, S, fp32_rounds ? &ob : o, 8, iters, refin);
    }
    CK(cudaMemcpyAsync(resid.data(), c->res.p, S * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
}

// One inner Krylov solve of A' x = b on the prepared operator, b and x in
// the caller's device memory (eels_krylov_solve_dev).  The context's stream
// waits for the caller's stream before reading b, and the caller's stream
// waits for the copy of x.
template <typename Rl>
void krylov_dev(eels_ctx* c, int solver, const void* b, void* x, int S, double eps, int max_iter, int* status,
                int* iters, cudaStream_t caller) {
    cudaStream_t st = c->stream;
    const int n3 = 3 * c->N;
    const int nblk = (n3 + RED_CHUNK - 1) / RED_CHUNK;
    const size_t kvec = (size_t)S * n3 * sizeof(cx<Rl>);
    for (auto& v : c->kv) v.ensure(kvec);
    c->part_a.ensure((size_t)S * std::max(nblk, 3 * c->L.Nx) * 4 * sizeof(double));
    c->part_b.ensure((size_t)S * nblk * 4 * sizeof(double));
    c->qmr.ensure((size_t)S * sizeof(QmrState));
    c->bicg.ensure((size_t)S * sizeof(BicgState));
    c->active.ensure(S * sizeof(int)); c->upd.ensure(S * sizeof(int)); c->counters.ensure(64);
    c->eps_sys.ensure(S * sizeof(double));
    cudaEvent_t ev;
    CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    struct EvGuard { cudaEvent_t e; ~EvGuard() { cudaEventDestroy(e); } } guard{ev};
    CK(cudaEventRecord(ev, caller));
    CK(cudaStreamWaitEvent(st, ev, 0));
    CK(cudaMemcpyAsync(c->kv[1].p, b, kvec, cudaMemcpyDeviceToDevice, st));   // rhs slot of every solver
    std::vector<int> one(S, 1), cnt(16, 0);
    cnt[0] = S;                                                             // systems still iterating
    std::vector<double> ev_eps(S, eps);
    h2d(c->active, one, st);
    h2d(c->counters, cnt, st);
    h2d(c->eps_sys, ev_eps, st);
    eels_opts o;
    eels_default_opts(&o);
    o.solver = solver;
    o.max_iter = max_iter;
    o.inner_max_iter = 0;
    inner_solve<Rl>(c, S, &o, eps);
    CK(cudaMemcpyAsync(x, c->kv[6].p, kvec, cudaMemcpyDeviceToDevice, st));
    std::vector<int> stv(S), itv(S);
    if (solver == EELS_BICGSTAB) {
        std::vector<BicgState> h(S);
        CK(cudaMemcpyAsync(h.data(), c->bicg.p, S * sizeof(BicgState), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (int i = 0; i < S; ++i) { stv[i] = h[i].status; itv[i] = h[i].iters; }
    } else if (solver == EELS_QMR2) {
        std::vector<Qmr2State> h(S);
        CK(cudaMemcpyAsync(h.data(), c->qmr.p, S * sizeof(Qmr2State), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (int i = 0; i < S; ++i) { stv[i] = h[i].status; itv[i] = h[i].iters; }
    } else {
        std::vector<QmrState> h(S);
        CK(cudaMemcpyAsync(h.data(), c->qmr.p, S * sizeof(QmrState), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (int i = 0; i < S; ++i) { stv[i] = h[i].status; itv[i] = h[i].iters; }
    }
    CK(cudaGetLastError());
    CK(cudaEventRecord(ev, st));
    CK(cudaStreamWaitEvent(caller, ev, 0));
    for (int i = 0; i < S; ++i) {
        // a system still marked running stopped at the host's iteration cap
        if (status) status[i] = stv[i] == 0 ? 2 : stv[i];
        if (iters) iters[i] = itv[i];
    }
}

int solve_impl(eels_ctx* c, const eels_opts* o, int n_energy, const double* energy_eV, int n_mat,
               const eels_c128* eps_p, const eels_c128* eps_h, int n_beam, const eels_beam* beams, double* p_eels,
               double* p_cl, double* p_ext, double* p_abs, eels_c128* p_out, eels_point_stats* stats) {
    if (!c->has_grid) throw Fail{EELS_E_NO_GRID, "eels_set_grid has not been called"};
    if (!o || n_energy <= 0 || n_beam <= 0 || !energy_eV || !eps_p || !eps_h || !beams || !p_eels)
        throw Fail{EELS_E_INVALID_ARG, "solve: NULL input or non-positive counts"};
    if (n_mat < c->max_mat || n_mat > EELS_MAX_MAT) throw Fail{EELS_E_INVALID_ARG, "n_mat does not cover the grid materials"};
    if (o->precision != EELS_FP64 && o->precision != EELS_MIXED) throw Fail{EELS_E_INVALID_ARG, "unknown precision"};
    if (o->solver != EELS_QMR && o->solver != EELS_BICGSTAB && o->solver != EELS_QMR2)
        throw Fail{EELS_E_INVALID_ARG, "unknown solver"};
    if (!(o->eps_it > 0) || o->max_iter <= 0) throw Fail{EELS_E_INVALID_ARG, "eps_it and max_iter must be positive"};
    if (p_cl && o->n_dir <= 0) throw Fail{EELS_E_INVALID_ARG, "p_cl requested with n_dir = 0"};
    if (o->interaction != EELS_INT_POINT && o->interaction != EELS_INT_IGT_SO)
        throw Fail{EELS_E_INVALID_ARG, "unknown interaction term"};
    if (o->polarizability != EELS_POL_CM && o->polarizability != EELS_POL_IGT_SO)
        throw Fail{EELS_E_INVALID_ARG, "unknown polarizability"};
    const BeamFrame frame = beam_frame(o->beam_dir);
    if (z_path(c, frame)) check_beams(c, n_beam, beams);
    else check_beams_dir(c, n_beam, beams, frame);
    CK(cudaSetDevice(c->device));
    cudaStream_t st = c->stream;
    const LatticeDev& L = c->L;
    const double d_m = c->d_nm * 1e-9;
    std::vector<EnergyPar> ep(n_energy);
    for (int e = 0; e < n_energy; ++e)
        ep[e] = energy_params(o->ekin_keV, energy_eV[e], cz(eps_h[e]), n_mat, eps_p + (size_t)e * n_mat, d_m,
                              o->polarizability);
    const bool fp64 = o->precision == EELS_FP64;
    const unsigned timeouts0 = wait_timeouts();
    // far-field directions
    std::vector<double> dirs_h, wts_h;
    if (p_cl) {
        if (c->dirs_n != o->n_dir) {
            if (!icosphere(o->n_dir, dirs_h, wts_h))
                throw Fail{EELS_E_INVALID_ARG, "n_dir must be 10*4^L+2 (icosphere vertex count)"};
            h2d(c->dirs, dirs_h, st);
            h2d(c->wts, wts_h, st);
            c->dirs_n = o->n_dir;
        }
    }
    // batch size
    const size_t per_sys = per_system_bytes(L, fp64);
    const size_t per_slot = per_slot_bytes(L);
    const size_t Mfull = (size_t)L.Mx * L.My * L.Mz;
    const size_t gslot = 6 * Mfull * sizeof(double2);
    int S_max = o->max_batch > 0 ? o->max_batch : 0;
    if (S_max <= 0) {
        size_t fr = 0, tot = 0;
        CK(cudaMemGetInfo(&fr, &tot));
        const size_t have = (size_t)(0.6 * (double)(fr + c->U.bytes + c->e64.bytes));
        S_max = (int)std::max<size_t>(1, have / (per_sys + per_slot + gslot / 8 + 1));
        S_max = std::min(S_max, 4096);
    }
    S_max = std::min(S_max, 21000);
    const int n_sys = n_energy * n_beam;
    c->spb = std::max(1, std::min(n_beam, c->spb_tuned > 0 ? c->spb_tuned : 16));
    std::vector<int> iters(n_sys, 0), refin(n_sys, 0);
    std::vector<double> resid(n_sys, 0.0);
    bool all_conv = true;
    for (int s0 = 0; s0 < n_sys; s0 += S_max) {
        const int S = std::min(S_max, n_sys - s0);
        const int e0 = s0 / n_beam, e1 = (s0 + S - 1) / n_beam + 1;
        const int n_slot = e1 - e0;
        const int n3 = 3 * c->N;
        const int nblk = (n3 + RED_CHUNK - 1) / RED_CHUNK;
        const size_t vec64 = (size_t)S * n3 * sizeof(double2);
        const size_t kvec = (size_t)S * n3 * (fp64 ? sizeof(double2) : sizeof(float2));
        c->e64.ensure(vec64); c->b64.ensure(vec64); c->x64.ensure(vec64); c->r64.ensure(vec64);
        c->y64.ensure(vec64); c->u64.ensure(vec64);
        c->u32.ensure((size_t)S * n3 * sizeof(float2));
        c->U.ensure((size_t)S * 3 * L.My * L.Nx * L.Mz * sizeof(double2));
        for (auto& b : c->kv) b.ensure(kvec);
        c->part_a.ensure((size_t)S * std::max(nblk, 3 * L.Nx) * 4 * sizeof(double));
        c->part_b.ensure((size_t)S * nblk * 4 * sizeof(double));
        c->qmr.ensure((size_t)S * sizeof(QmrState));
        c->bicg.ensure((size_t)S * sizeof(BicgState));
        c->active.ensure(S * sizeof(int)); c->upd.ensure(S * sizeof(int)); c->outer.ensure(S * sizeof(int));
        c->counters.ensure(64);
        c->res.ensure(S * sizeof(double)); c->rnorm.ensure(S * sizeof(double)); c->eps_sys.ensure(S * sizeof(double));
        c->Dr64.ensure((size_t)n_slot * 6 * L.Hx * L.Hy * L.Hz * sizeof(double2));
        c->Dr32.ensure((size_t)n_slot * 6 * L.Hx * L.Hy * L.Hz * sizeof(float2));
        c->Dx32.ensure((size_t)n_slot * 6 * L.Hx * L.Hy * L.Hz * sizeof(float2));
        // D-hat for the batch energies, in chunks that fit ~1/8 of the system budget
        const int gchunk = (int)std::max<size_t>(1, std::min<size_t>(n_slot, (size_t)std::max(1, S) * per_sys / 8 / gslot + 1));
        c->G.ensure(gchunk * gslot);
        std::vector<double2> kap_slot(n_slot);
        for (int e = e0; e < e1; ++e) kap_slot[e - e0] = d2(ep[e].kappa);
        h2d(c->kappa_slot, kap_slot, st);
        for (int q0 = 0; q0 < n_slot; q0 += gchunk) {
            const int nq = std::min(gchunk, n_slot - q0);
            const size_t hs = (size_t)6 * L.Hx * L.Hy * L.Hz;
            launch_dhat_build(dhat_lattice(c, o->interaction), nq, c->kappa_slot.as<double2>() + q0, c->G.as<double2>(),
                              c->Dr64.as<double2>() + q0 * hs,
                              c->Dr32.as<float2>() + q0 * hs, st, c->Dx32.as<float2>() + q0 * hs);
        }
        CK(cudaGetLastError());
        // per-system parameters
        std::vector<SysField> sf(S);
        std::vector<double2> coef((size_t)S * EELS_MAX_MAT), diag((size_t)S * EELS_MAX_MAT, make_double2(1, 0));
        std::vector<double> wabs((size_t)S * EELS_MAX_MAT, 0.0), wdv(S);
        std::vector<int> slot(S);
        std::vector<double2> kap(S);
        for (int s = 0; s < S; ++s) {
            const int g = s0 + s, e = g / n_beam, b = g % n_beam;
            const EnergyPar& p = ep[e];
            sf[s].kt = d2(p.wdv / p.gamma);
            sf[s].inv_gamma = d2(1.0 / p.gamma);
            sf[s].pref_unit = d2(p.pref_unit);
            sf[s].wdv = p.wdv;
            set_beam(sf[s], frame, beams[b], c);
            for (int m = 0; m < EELS_MAX_MAT; ++m) {
                coef[(size_t)s * EELS_MAX_MAT + m] = m < n_mat ? d2(p.sa[m]) : make_double2(0, 0);
                wabs[(size_t)s * EELS_MAX_MAT + m] = m < n_mat ? p.wabs[m] : 0.0;
            }
            wdv[s] = p.wdv;
            slot[s] = e - e0;
            kap[s] = d2(p.kappa);
        }
        h2d(c->sysf, sf, st); h2d(c->coef, coef, st); h2d(c->diag, diag, st); h2d(c->wabs, wabs, st);
        h2d(c->wdv, wdv, st); h2d(c->slot, slot, st); h2d(c->kappa_sys, kap, st);
        launch_incident_field(L, S, c->sysf.as<SysField>(), z_path(c, frame), c->e64.as<double2>(), st);
        launch_rhs_init(L, S, c->e64.as<double2>(), c->coef.as<double2>(), c->b64.as<double2>(), c->x64.as<double2>(),
                        c->r64.as<double2>(), st);
        // y = A x for x = 0: refinement rounds recompute y only for the systems they update
        CK(cudaMemsetAsync(c->y64.p, 0, (size_t)S * 3 * c->N * sizeof(double2), st));
        CK(cudaGetLastError());
        std::vector<int> it_b(S, 0), rf_b(S, 0);
        std::vector<double> rs_b(S, 0.0);
        if (!c->tuned) {
            // first solve on this lattice: time the x-pass tile widths on this
            // batch (the x pass only scrambles the FFT scratch), before any
            // inner-loop graph is captured; FP64 on a few systems only
            // (the register-resident FP32 x pass: how U moves and how many beams
            // of an energy a block takes are timed instead of the tile width)
            if (xpass_reg_supported(L)) {
                CK(cudaMemsetAsync(c->U.p, 0, (size_t)S * 3 * L.My * L.Nx * L.Mz * sizeof(float2), st));
                int mode = 0, spb = 1;
                autotune_xreg(L, mv_args<float>(c, S, c->u32.as<float2>(), c->kv[5].as<float2>(), c->Dr32.as<float2>(),
                                                 nullptr, true),
                              c->spb, st, &mode, &spb, &c->xreg_log);
                c->L.xmode = mode;
                c->spb_tuned = spb;
                c->spb = std::min(c->spb, spb);
            }
            c->L.xw32 = xpass_reg_supported(L) ? 16
                                               : autotune_xpass<float>(L, mv_args<float>(c, S, c->u32.as<float2>(),
                                                                                          c->kv[5].as<float2>(),
                                                                                          c->Dr32.as<float2>(), nullptr,
                                                                                          true), st);
            c->L.xw64 = autotune_xpass<double>(L, mv_args<double>(c, std::min(S, 8), c->x64.as<double2>(),
                                                                   c->y64.as<double2>(), c->Dr64.as<double2>(),
                                                                   nullptr, true), st);
            c->tuned = true;
            c->tune_cache[c->shape_key()] = {c->L.xw32, c->L.xw64, c->L.xmode, c->spb_tuned, c->xreg_log};
        }
        refine_batch(c, S, o, fp64, it_b, rf_b, rs_b);
        // losses
        const int lblk = std::max(1, std::min(64, (c->N + 2047) / 2048));
        c->lpart.ensure((size_t)S * lblk * 8 * sizeof(double));
        c->lsums.ensure((size_t)S * 5 * sizeof(double));
        launch_losses(L, S, c->e64.as<double2>(), c->x64.as<double2>(), c->coef.as<double2>(), c->wabs.as<double>(),
                      c->wdv.as<double>(), c->sysf.as<SysField>(), c->lpart.as<double>(), lblk, c->lsums.as<double>(), st);
        std::vector<double> ls((size_t)S * 5), fs(S, 0.0);
        CK(cudaMemcpyAsync(ls.data(), c->lsums.p, ls.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        if (p_cl || p_out)
            launch_scaled_dipoles(L, S, c->x64.as<double2>(), c->coef.as<double2>(), c->u64.as<double2>(),
                                  c->u32.as<float2>(), st);
        if (p_cl) {
            const int nbf = (o->n_dir + 127) / 128;
            c->fpart.ensure((size_t)S * nbf * sizeof(double));
            c->fsums.ensure((size_t)S * sizeof(double));
            if (fp64)
                launch_farfield<double>(L, S, c->u64.as<double2>(), c->kappa_sys.as<double2>(), c->dirs.as<double>(),
                                        c->wts.as<double>(), o->n_dir, c->fpart.as<double>(), c->fsums.as<double>(), st);
            else
                launch_farfield<float>(L, S, c->u32.as<float2>(), c->kappa_sys.as<double2>(), c->dirs.as<double>(),
                                       c->wts.as<double>(), o->n_dir, c->fpart.as<double>(), c->fsums.as<double>(), st);
            CK(cudaMemcpyAsync(fs.data(), c->fsums.p, S * sizeof(double), cudaMemcpyDeviceToHost, st));
        }
        std::vector<double2> uh;
        if (p_out) {
            uh.resize((size_t)S * n3);
            CK(cudaMemcpyAsync(uh.data(), c->u64.p, uh.size() * sizeof(double2), cudaMemcpyDeviceToHost, st));
        }
        CK(cudaStreamSynchronize(st));
        CK(cudaGetLastError());
        for (int s = 0; s < S; ++s) {
            const int g = s0 + s, e = g / n_beam;
            const EnergyPar& p = ep[e];
            const double d3 = d_m * d_m * d_m;
            const double f = 4.0 * kEps0 * d3 * p.scale * p.scale / (kHbar * kHbar) * kE;
            const cd sa(ls[s * 5 + 0], ls[s * 5 + 1]), sx(ls[s * 5 + 2], ls[s * 5 + 3]);
            p_eels[g] = -f * (p.eps_h * sa).imag();
            if (p_ext) p_ext[g] = f * (p.eps_h * sx).imag();
            if (p_abs) p_abs[g] = f * p.eps_h.real() * ls[s * 5 + 4];
            if (p_cl) {
                const double ak = std::abs(p.kappa);
                p_cl[g] = p.m_h.real() * kEps0 * kC * ak * ak * ak * ak * d_m * d_m * p.scale * p.scale * fs[s] /
                          (kPi * kHbar * kHbar * p.omega) * kE;
            }
            if (p_out) {
                const cd fac = 4.0 * kPi * kEps0 * p.eps_h * d3 * p.scale;
                for (int i = 0; i < c->N; ++i)
                    for (int a = 0; a < 3; ++a) {
                        const double2 u = uh[(size_t)s * n3 + (size_t)a * c->N + i];
                        const cd v = fac * cd(u.x, u.y);
                        p_out[((size_t)g * c->N + c->abi_of[i]) * 3 + a] = {v.real(), v.imag()};
                    }
            }
            const bool conv = rs_b[s] <= o->eps_it;
            all_conv = all_conv && conv;
            if (stats) {
                stats[g].iters = it_b[s];
                stats[g].refinements = rf_b[s];
                stats[g].residual = rs_b[s];
                stats[g].converged = conv ? 1 : 0;
            }
        }
    }
    if (wait_timeouts() != timeouts0)
        throw Fail{EELS_E_TIMEOUT, "a bounded device-side wait expired: results of this solve are incomplete"};
    return all_conv ? EELS_OK : EELS_E_NOT_CONVERGED;
}

// Entry points that take the caller's device pointers and stream run on the
// caller's current device: it must be the context's, whose D-hat, lattice
// tables and scratch the kernels read.
void require_current_device(const eels_ctx* c) {
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) {
        cudaGetLastError();
        throw Fail{EELS_E_CUDA, "cudaGetDevice failed"};
    }
    if (cur != c->device)
        throw Fail{EELS_E_INVALID_ARG, "the current device (" + std::to_string(cur) + ") is not the context's device (" +
                                           std::to_string(c->device) + "): make it current before the call"};
}

template <typename F> int guarded(eels_ctx* c, F&& f) {
    try {
        if (c) c->err.clear();
        return f();
    } catch (const Fail& e) {
        set_err(c, e.msg);
        return e.code;
    } catch (const std::exception& e) {
        set_err(c, e.what());
        return EELS_E_CUDA;
    }
}

}  // namespace

// =========================================================================
// C ABI
// =========================================================================
extern "C" {

void eels_default_opts(eels_opts* o) {
    if (!o) return;
    o->ekin_keV = 100.0;
    o->precision = EELS_MIXED;
    o->solver = EELS_QMR2;
    o->eps_it = 1e-8;
    o->eps_inner = 1e-5;
    o->max_iter = 20000;
    o->n_dir = 2562;
    o->max_batch = 0;
    o->inner_max_iter = 2000;
    o->beam_dir[0] = 0.0;
    o->beam_dir[1] = 0.0;
    o->beam_dir[2] = 1.0;
    o->interaction = EELS_INT_POINT;
    o->polarizability = EELS_POL_CM;
    o->device_loop = 0;
}

int eels_set_interaction(eels_ctx* c, int interaction, int polarizability) {
    if (!c) return EELS_E_INVALID_ARG;
    return guarded(c, [&] {
        if (interaction != EELS_INT_POINT && interaction != EELS_INT_IGT_SO)
            throw Fail{EELS_E_INVALID_ARG, "unknown interaction term"};
        if (polarizability != EELS_POL_CM && polarizability != EELS_POL_IGT_SO)
            throw Fail{EELS_E_INVALID_ARG, "unknown polarizability"};
        c->interaction = interaction;
        c->polarizability = polarizability;
        return EELS_OK;
    });
}

int eels_create(eels_ctx** out, int device, void* cuda_stream) {
    if (!out) return EELS_E_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return EELS_E_CUDA;
    }
    auto* c = new eels_ctx();
    c->device = device;
    if (cudaSetDevice(device) != cudaSuccess) { delete c; return EELS_E_CUDA; }
    // shared-memory opt-in for every kernel instance, once per device and
    // outside any stream capture
    static std::mutex mu;
    static std::vector<int> prepared;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (std::find(prepared.begin(), prepared.end(), device) == prepared.end()) {
            prepare_kernels();
            prepared.push_back(device);
        }
    }
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) { delete c; return EELS_E_CUDA; }
        c->own_stream = true;
    }
    if (cudaMallocHost(&c->pinned, 64) != cudaSuccess) {
        if (c->own_stream) cudaStreamDestroy(c->stream);
        delete c;
        return EELS_E_OOM;
    }
    for (DevBuf* b : c->buffers()) b->sp = &c->stream;
    *out = c;
    return EELS_OK;
}

void eels_destroy(eels_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    if (c->graph) cudaGraphExecDestroy(c->graph);
    for (DevBuf* b : c->buffers()) b->release();
    cudaStreamSynchronize(c->stream);
    if (c->pinned) cudaFreeHost(c->pinned);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

const char* eels_last_error(const eels_ctx* c) { return c ? c->err.c_str() : ""; }

int eels_set_grid(eels_ctx* c, const eels_grid* g) {
    if (!c) return EELS_E_INVALID_ARG;
    return guarded(c, [&] { set_grid(c, g); return EELS_OK; });
}

int eels_num_dipoles(const eels_ctx* c) { return (c && c->has_grid) ? c->N : 0; }

int eels_tile_widths(const eels_ctx* c, int* xw32, int* xw64) {
    if (!c || !xw32 || !xw64) return EELS_E_INVALID_ARG;
    if (!c->has_grid) return EELS_E_NO_GRID;
    *xw32 = c->L.xw32;
    *xw64 = c->L.xw64;
    return EELS_OK;
}

int eels_tuned_xpass(const eels_ctx* c, int* mode, int* spb) {
    if (!c || !mode || !spb) return EELS_E_INVALID_ARG;
    if (!c->has_grid) return EELS_E_NO_GRID;
    *mode = c->L.xmode;
    *spb = c->spb_tuned;
    return EELS_OK;
}

int eels_xpass_timings(const eels_ctx* c, int cap, int* n, int* mode, int* spb, float* ms) {
    if (!c || !n || cap < 0 || (cap > 0 && (!mode || !spb || !ms))) return EELS_E_INVALID_ARG;
    if (!c->has_grid) return EELS_E_NO_GRID;
    *n = (int)c->xreg_log.size();
    for (int i = 0; i < cap && i < *n; ++i) {
        mode[i] = (int)c->xreg_log[i][0];
        spb[i] = (int)c->xreg_log[i][1];
        ms[i] = c->xreg_log[i][2];
    }
    return EELS_OK;
}

int eels_padded_dims(const eels_ctx* c, int* mx, int* my, int* mz) {
    if (!c || !c->has_grid) return EELS_E_NO_GRID;
    if (mx) *mx = c->L.Mx;
    if (my) *my = c->L.My;
    if (mz) *mz = c->L.Mz;
    return EELS_OK;
}

int eels_solve(eels_ctx* c, const eels_opts* o, int n_energy, const double* energy_eV, int n_mat,
               const eels_c128* eps_p, const eels_c128* eps_h, int n_beam, const eels_beam* beams, double* p_eels,
               double* p_cl, double* p_ext, double* p_abs, eels_c128* p_out, eels_point_stats* stats) {
    if (!c) return EELS_E_INVALID_ARG;
    return guarded(c, [&] {
        return solve_impl(c, o, n_energy, energy_eV, n_mat, eps_p, eps_h, n_beam, beams, p_eels, p_cl, p_ext, p_abs,
                          p_out, stats);
    });
}

int eels_query_footprint(const eels_grid* g, const eels_opts* o, int n_systems, size_t* bytes) {
    if (!g || !o || !bytes || n_systems <= 0 || g->nx <= 0 || g->ny <= 0 || g->nz <= 0 || !g->occ) return EELS_E_INVALID_ARG;
    LatticeDev L{};
    L.Nx = g->nx; L.Ny = g->ny; L.Nz = g->nz;
    size_t n = 0;
    for (size_t i = 0; i < (size_t)g->nx * g->ny * g->nz; ++i) n += g->occ[i] != 0;
    L.N = (int)n;
    L.Mx = pad_len_x(g->nx); L.My = good_fft_len(g->ny); L.Mz = good_fft_len(g->nz);
    L.Hx = L.Mx / 2 + 1; L.Hy = L.My / 2 + 1; L.Hz = L.Mz / 2 + 1;
    const size_t Mfull = (size_t)L.Mx * L.My * L.Mz;
    *bytes = (size_t)n_systems * (per_system_bytes(L, o->precision == EELS_FP64) + per_slot_bytes(L)) +
             6 * Mfull * sizeof(double2) + (size_t)L.Nx * L.Ny * L.Nz * 4 + n * 8;
    return EELS_OK;
}

int eels_bessel_k01_dev(const eels_c128* z, eels_c128* k0, eels_c128* k1, int n, void* stream) {
    if (n < 0 || (n > 0 && (!z || !k0 || !k1))) return EELS_E_INVALID_ARG;
    launch_bessel(reinterpret_cast<const double2*>(z), reinterpret_cast<double2*>(k0), reinterpret_cast<double2*>(k1), n,
                  (cudaStream_t)stream);
    return cudaGetLastError() == cudaSuccess ? EELS_OK : EELS_E_CUDA;
}

int eels_incident_field_dir(eels_ctx* c, double ekin_keV, double energy_eV, eels_c128 eps_h, eels_beam beam,
                            const double* beam_dir, eels_c128* e_inc, eels_c128* e_aux) {
    if (!c) return EELS_E_INVALID_ARG;
    return guarded(c, [&] {
        if (!c->has_grid) throw Fail{EELS_E_NO_GRID, "eels_set_grid has not been called"};
        const double zdir[3] = {0.0, 0.0, 1.0};
        const BeamFrame frame = beam_frame(beam_dir ? beam_dir : zdir);
        if (z_path(c, frame)) check_beams(c, 1, &beam);
        else check_beams_dir(c, 1, &beam, frame);
        CK(cudaSetDevice(c->device));
        const double d_m = c->d_nm * 1e-9;
        eels_c128 one{1.0, 0.0};
        EnergyPar p = energy_params(ekin_keV, energy_eV, cz(eps_h), 1, &one, d_m);
        SysField sf;
        sf.kt = d2(p.wdv / p.gamma); sf.inv_gamma = d2(1.0 / p.gamma); sf.pref_unit = d2(p.pref_unit);
        sf.wdv = p.wdv;
        set_beam(sf, frame, beam, c);
        std::vector<SysField> sv(1, sf);
        cudaStream_t st = c->stream;
        h2d(c->sysf, sv, st);
        const size_t n3 = (size_t)3 * c->N;
        c->e64.ensure(n3 * sizeof(double2));
        c->y64.ensure(n3 * sizeof(double2));
        launch_incident_field(c->L, 1, c->sysf.as<SysField>(), z_path(c, frame), c->e64.as<double2>(), st);
        launch_aux_field(c->L, 1, c->sysf.as<SysField>(), c->e64.as<double2>(), c->y64.as<double2>(), st);
        std::vector<double2> h(n3), ha(n3);
        CK(cudaMemcpyAsync(h.data(), c->e64.p, n3 * sizeof(double2), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(ha.data(), c->y64.p, n3 * sizeof(double2), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        CK(cudaGetLastError());
        for (int i = 0; i < c->N; ++i)
            for (int a = 0; a < 3; ++a) {
                const double2 v = h[(size_t)a * c->N + i], va = ha[(size_t)a * c->N + i];
                if (e_inc) e_inc[(size_t)c->abi_of[i] * 3 + a] = {v.x * p.scale, v.y * p.scale};
                if (e_aux) e_aux[(size_t)c->abi_of[i] * 3 + a] = {va.x * p.scale, va.y * p.scale};
            }
        return EELS_OK;
    });
}

int eels_incident_field(eels_ctx* c, double ekin_keV, double energy_eV, eels_c128 eps_h, eels_beam beam,
                        eels_c128* e_inc, eels_c128* e_aux) {
    return eels_incident_field_dir(c, ekin_keV, energy_eV, eps_h, beam, nullptr, e_inc, e_aux);
}

int eels_apply_matrix(eels_ctx* c, int precision, double energy_eV, int n_mat, const eels_c128* eps_p, eels_c128 eps_h,
                      int n_vec, const eels_c128* x, eels_c128* y) {
    if (!c) return EELS_E_INVALID_ARG;
    return guarded(c, [&] {
        if (!c->has_grid) throw Fail{EELS_E_NO_GRID, "eels_set_grid has not been called"};
        if (n_vec <= 0 || !x || !y || !eps_p || n_mat < c->max_mat || n_mat > EELS_MAX_MAT)
            throw Fail{EELS_E_INVALID_ARG, "apply_matrix: bad arguments"};
        CK(cudaSetDevice(c->device));
        cudaStream_t st = c->stream;
        const LatticeDev& L = c->L;
        const double d_m = c->d_nm * 1e-9;
        EnergyPar p = energy_params(100.0, energy_eV, cz(eps_h), n_mat, eps_p, d_m, c->polarizability);
        const int S = n_vec, n3 = 3 * c->N;
        const size_t hs = (size_t)6 * L.Hx * L.Hy * L.Hz;
        c->Dr64.ensure(hs * sizeof(double2));
        c->Dr32.ensure(hs * sizeof(float2));
        c->Dx32.ensure(hs * sizeof(float2));
        c->G.ensure((size_t)6 * L.Mx * L.My * L.Mz * sizeof(double2));
        std::vector<double2> ks(1, d2(p.kappa));
        h2d(c->kappa_slot, ks, st);
        launch_dhat_build(dhat_lattice(c, c->interaction), 1, c->kappa_slot.as<double2>(), c->G.as<double2>(),
                          c->Dr64.as<double2>(), c->Dr32.as<float2>(), st,
                          c->Dx32.as<float2>());
        std::vector<double2> coef((size_t)S * EELS_MAX_MAT, make_double2(1, 0)), diag((size_t)S * EELS_MAX_MAT);
        for (int s = 0; s < S; ++s)
            for (int m = 0; m < EELS_MAX_MAT; ++m) diag[(size_t)s * EELS_MAX_MAT + m] = m < n_mat ? d2(p.alpha_inv[m]) : make_double2(0, 0);
        std::vector<int> slot(S, 0);
        c->spb = std::min(S, 16);
        h2d(c->coef, coef, st); h2d(c->diag, diag, st); h2d(c->slot, slot, st);
        std::vector<double2> xh((size_t)S * n3);
        for (int s = 0; s < S; ++s)
            for (int i = 0; i < c->N; ++i)
                for (int a = 0; a < 3; ++a) {
                    const eels_c128 v = x[((size_t)s * c->N + c->abi_of[i]) * 3 + a];
                    xh[(size_t)s * n3 + (size_t)a * c->N + i] = make_double2(v.re, v.im);
                }
        c->x64.ensure(xh.size() * sizeof(double2));
        c->y64.ensure(xh.size() * sizeof(double2));
        c->U.ensure((size_t)S * 3 * L.My * L.Nx * L.Mz * sizeof(double2));
        CK(cudaMemcpyAsync(c->x64.p, xh.data(), xh.size() * sizeof(double2), cudaMemcpyHostToDevice, st));
        std::vector<double2> yh(xh.size());
        if (precision == EELS_FP64) {
            MatvecArgs<double> a = mv_args<double>(c, S, c->x64.as<double2>(), c->y64.as<double2>(), c->Dr64.as<double2>(), nullptr, false);
            launch_matvec<double>(L, a, st);
            CK(cudaMemcpyAsync(yh.data(), c->y64.p, yh.size() * sizeof(double2), cudaMemcpyDeviceToHost, st));
        } else {
            c->u32.ensure(xh.size() * sizeof(float2));
            c->kv[5].ensure(xh.size() * sizeof(float2));
            launch_to_f32(xh.size(), c->x64.as<double2>(), c->u32.as<float2>(), st);
            MatvecArgs<float> a = mv_args<float>(c, S, c->u32.as<float2>(), c->kv[5].as<float2>(), c->Dr32.as<float2>(), nullptr, false);
            launch_matvec<float>(L, a, st);
            std::vector<float2> yf(xh.size());
            CK(cudaMemcpyAsync(yf.data(), c->kv[5].p, yf.size() * sizeof(float2), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            for (size_t i = 0; i < yf.size(); ++i) yh[i] = make_double2(yf[i].x, yf[i].y);
        }
        CK(cudaStreamSynchronize(st));
        CK(cudaGetLastError());
        const double inv_d3 = 1.0 / (d_m * d_m * d_m);
        for (int s = 0; s < S; ++s)
            for (int i = 0; i < c->N; ++i)
                for (int a = 0; a < 3; ++a) {
                    const double2 v = yh[(size_t)s * n3 + (size_t)a * c->N + i];
                    y[((size_t)s * c->N + c->abi_of[i]) * 3 + a] = {v.x * inv_d3, v.y * inv_d3};
                }
        return EELS_OK;
    });
}

int eels_prepare_operator(eels_ctx* c, int n_energy, const double* energy_eV, int n_mat, const eels_c128* eps_p,
                          const eels_c128* eps_h) {
    if (!c) return EELS_E_INVALID_ARG;
    return guarded(c, [&] {
        if (!c->has_grid) throw Fail{EELS_E_NO_GRID, "eels_set_grid has not been called"};
        if (n_energy <= 0 || !energy_eV || !eps_p || !eps_h || n_mat < c->max_mat || n_mat > EELS_MAX_MAT)
            throw Fail{EELS_E_INVALID_ARG, "prepare_operator: bad arguments"};
        CK(cudaSetDevice(c->device));
        cudaStream_t st = c->stream;
        const LatticeDev& L = c->L;
        const double d_m = c->d_nm * 1e-9;
        const int S = n_energy;
        const size_t hs = (size_t)6 * L.Hx * L.Hy * L.Hz;
        c->Dr64.ensure(S * hs * sizeof(double2));
        c->Dr32.ensure(S * hs * sizeof(float2));
        c->Dx32.ensure(S * hs * sizeof(float2));
        const size_t gslot = (size_t)6 * L.Mx * L.My * L.Mz * sizeof(double2);
        c->G.ensure(gslot);
        std::vector<double2> kap, coef((size_t)S * EELS_MAX_MAT), diag((size_t)S * EELS_MAX_MAT, make_double2(1, 0));
        std::vector<int> slot(S);
        // consecutive systems with the same energy and permittivities share one
        // D-hat slot (the beams of one energy)
        int run = 0, max_run = 1;
        for (int e = 0; e < S; ++e) {
            EnergyPar p = energy_params(100.0, energy_eV[e], cz(eps_h[e]), n_mat, eps_p + (size_t)e * n_mat, d_m,
                                        c->polarizability);
            const bool same = e > 0 && energy_eV[e] == energy_eV[e - 1] && eps_h[e].re == eps_h[e - 1].re &&
                              eps_h[e].im == eps_h[e - 1].im &&
                              std::memcmp(eps_p + (size_t)e * n_mat, eps_p + (size_t)(e - 1) * n_mat,
                                          n_mat * sizeof(eels_c128)) == 0;
            if (!same) kap.push_back(d2(p.kappa));
            run = same ? run + 1 : 1;
            max_run = std::max(max_run, run);
            slot[e] = (int)kap.size() - 1;
            for (int m = 0; m < EELS_MAX_MAT; ++m) coef[(size_t)e * EELS_MAX_MAT + m] = m < n_mat ? d2(p.sa[m]) : make_double2(0, 0);
        }
        h2d(c->kappa_slot, kap, st);
        for (size_t e = 0; e < kap.size(); ++e)
            launch_dhat_build(dhat_lattice(c, c->interaction), 1, c->kappa_slot.as<double2>() + e, c->G.as<double2>(),
                              c->Dr64.as<double2>() + e * hs,
                              c->Dr32.as<float2>() + e * hs, st, c->Dx32.as<float2>() + e * hs);
        c->spb = std::min(max_run, 16);
        h2d(c->coef, coef, st); h2d(c->diag, diag, st); h2d(c->slot, slot, st);
        c->U.ensure((size_t)S * 3 * L.My * L.Nx * L.Mz * sizeof(double2));
        CK(cudaStreamSynchronize(st));
        CK(cudaGetLastError());
        c->op_systems = S;
        return EELS_OK;
    });
}

int eels_matvec_dev(eels_ctx* c, int precision, const void* x, void* y, int n_sys, void* stream) {
    if (!c) return EELS_E_INVALID_ARG;
    return guarded(c, [&] {
        if (!c->has_grid) throw Fail{EELS_E_NO_GRID, "eels_set_grid has not been called"};
        if (n_sys <= 0 || n_sys > c->op_systems || !x || !y)
            throw Fail{EELS_E_INVALID_ARG, "matvec_dev: n_sys must be in [1, prepared systems]"};
        require_current_device(c);
        cudaStream_t st = (cudaStream_t)stream;
        if (precision == EELS_FP64) {
            MatvecArgs<double> a = mv_args<double>(c, n_sys, (const double2*)x, (double2*)y, c->Dr64.as<double2>(), nullptr, true);
            launch_matvec<double>(c->L, a, st);
        } else {
            MatvecArgs<float> a = mv_args<float>(c, n_sys, (const float2*)x, (float2*)y, c->Dr32.as<float2>(), nullptr, true);
            launch_matvec<float>(c->L, a, st);
        }
        CK(cudaGetLastError());
        return EELS_OK;
    });
}

int eels_krylov_solve_dev(eels_ctx* c, int precision, int solver, const void* b, void* x, int n_sys, double eps,
                          int max_iter, int* status, int* iters, void* stream) {
    if (!c) return EELS_E_INVALID_ARG;
    return guarded(c, [&] {
        if (!c->has_grid) throw Fail{EELS_E_NO_GRID, "eels_set_grid has not been called"};
        if (n_sys <= 0 || n_sys > c->op_systems || !b || !x || b == x)
            throw Fail{EELS_E_INVALID_ARG, "krylov_solve_dev: n_sys must be in [1, prepared systems], b and x distinct"};
        if (!(eps > 0) || max_iter <= 0) throw Fail{EELS_E_INVALID_ARG, "krylov_solve_dev: eps and max_iter must be positive"};
        if (precision != EELS_FP64 && precision != EELS_MIXED) throw Fail{EELS_E_INVALID_ARG, "unknown precision"};
        if (solver != EELS_QMR && solver != EELS_BICGSTAB && solver != EELS_QMR2)
            throw Fail{EELS_E_INVALID_ARG, "unknown solver"};
        require_current_device(c);
        if (precision == EELS_FP64)
            krylov_dev<double>(c, solver, b, x, n_sys, eps, max_iter, status, iters, (cudaStream_t)stream);
        else
            krylov_dev<float>(c, solver, b, x, n_sys, eps, max_iter, status, iters, (cudaStream_t)stream);
        return EELS_OK;
    });
}

int eels_solve_dev(eels_ctx* c, const eels_opts* o, int n_energy, const double* energy_eV, int n_mat,
                   const eels_c128* eps_p, const eels_c128* eps_h, int n_beam, const eels_beam* beams,
                   double* p_eels, double* p_cl, double* p_ext, double* p_abs, eels_c128* p_out,
                   eels_point_stats* stats, void* stream) {
    if (!c) return EELS_E_INVALID_ARG;
    return guarded(c, [&] {
        if (!o || n_energy <= 0 || n_beam <= 0 || n_mat <= 0 || !energy_eV || !eps_p || !eps_h || !beams || !p_eels)
            throw Fail{EELS_E_INVALID_ARG, "solve_dev: NULL input or non-positive counts"};
        require_current_device(c);
        // every array argument must be device memory of the context's device
        const void* ptrs[] = {energy_eV, eps_p, eps_h, beams, p_eels, p_cl, p_ext, p_abs, p_out, stats};
        for (const void* q : ptrs) {
            if (!q) continue;
            cudaPointerAttributes at{};
            if (cudaPointerGetAttributes(&at, q) != cudaSuccess) {
                cudaGetLastError();
                throw Fail{EELS_E_INVALID_ARG, "solve_dev: an array argument is not CUDA memory"};
            }
            if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
                throw Fail{EELS_E_INVALID_ARG, "solve_dev: array arguments must be device memory"};
            if (at.type == cudaMemoryTypeDevice && at.device != c->device)
                throw Fail{EELS_E_INVALID_ARG, "solve_dev: an array argument lives on another device"};
        }
        cudaStream_t caller = (cudaStream_t)stream;
        const size_t ne = (size_t)n_energy, np = (size_t)n_energy * n_beam;
        // inputs: read in the caller's stream order
        std::vector<double> e_h(ne);
        std::vector<eels_c128> ep_h(ne * n_mat), eh_h(ne);
        std::vector<eels_beam> b_h(n_beam);
        CK(cudaMemcpyAsync(e_h.data(), energy_eV, ne * sizeof(double), cudaMemcpyDeviceToHost, caller));
        CK(cudaMemcpyAsync(ep_h.data(), eps_p, ep_h.size() * sizeof(eels_c128), cudaMemcpyDeviceToHost, caller));
        CK(cudaMemcpyAsync(eh_h.data(), eps_h, ne * sizeof(eels_c128), cudaMemcpyDeviceToHost, caller));
        CK(cudaMemcpyAsync(b_h.data(), beams, n_beam * sizeof(eels_beam), cudaMemcpyDeviceToHost, caller));
        CK(cudaStreamSynchronize(caller));
        std::vector<double> pe(np), pc(p_cl ? np : 0), px(p_ext ? np : 0), pa(p_abs ? np : 0);
        std::vector<eels_c128> po(p_out ? np * (size_t)c->N * 3 : 0);
        std::vector<eels_point_stats> sv(np);
        const int code = solve_impl(c, o, n_energy, e_h.data(), n_mat, ep_h.data(), eh_h.data(), n_beam, b_h.data(),
                                    pe.data(), p_cl ? pc.data() : nullptr, p_ext ? px.data() : nullptr,
                                    p_abs ? pa.data() : nullptr, p_out ? po.data() : nullptr, sv.data());
        // outputs: written in the caller's stream order; the call returns once they are in place
        CK(cudaMemcpyAsync(p_eels, pe.data(), np * sizeof(double), cudaMemcpyHostToDevice, caller));
        if (p_cl) CK(cudaMemcpyAsync(p_cl, pc.data(), np * sizeof(double), cudaMemcpyHostToDevice, caller));
        if (p_ext) CK(cudaMemcpyAsync(p_ext, px.data(), np * sizeof(double), cudaMemcpyHostToDevice, caller));
        if (p_abs) CK(cudaMemcpyAsync(p_abs, pa.data(), np * sizeof(double), cudaMemcpyHostToDevice, caller));
        if (p_out) CK(cudaMemcpyAsync(p_out, po.data(), po.size() * sizeof(eels_c128), cudaMemcpyHostToDevice, caller));
        if (stats) CK(cudaMemcpyAsync(stats, sv.data(), np * sizeof(eels_point_stats), cudaMemcpyHostToDevice, caller));
        CK(cudaStreamSynchronize(caller));
        return code;
    });
}

long long eels_kernel_launches(void) { return g_kernel_launches.load(); }

}  // extern "C"

int eels_internal_device(const eels_ctx* c) { return c ? c->device : -1; }

// Launch the prepared operator with caller-provided FFT scratch (used by
// eels_matvec_dev_noalloc, which owns a fixed array).  Allocates nothing.
int eels_internal_matvec_with_scratch(eels_ctx* c, int precision, const void* x, void* y, int n_sys, void* stream,
                                      void* scratch, size_t scratch_bytes) {
    if (!c) return EELS_E_INVALID_ARG;
    return guarded(c, [&] {
        if (!c->has_grid) throw Fail{EELS_E_NO_GRID, "eels_set_grid has not been called"};
        if (n_sys <= 0 || n_sys > c->op_systems || !x || !y)
            throw Fail{EELS_E_INVALID_ARG, "matvec: n_sys must be in [1, prepared systems]"};
        require_current_device(c);
        const LatticeDev& L = c->L;
        const size_t elem = precision == EELS_FP64 ? sizeof(double2) : sizeof(float2);
        const size_t need = (size_t)n_sys * 3 * L.My * L.Nx * L.Mz * elem;
        if (need > scratch_bytes)
            throw Fail{EELS_E_UNSUPPORTED, "eels_matvec_dev_noalloc: " + std::to_string(n_sys) + " systems need " +
                                               std::to_string(need) + " bytes of FFT scratch, more than the fixed " +
                                               std::to_string(scratch_bytes) + "-byte array; pass fewer systems per call"};
        cudaStream_t st = (cudaStream_t)stream;
        if (precision == EELS_FP64) {
            MatvecArgs<double> a = mv_args<double>(c, n_sys, (const double2*)x, (double2*)y, c->Dr64.as<double2>(), nullptr, true);
            a.U = reinterpret_cast<double2*>(scratch);
            launch_matvec<double>(L, a, st);
        } else {
            MatvecArgs<float> a = mv_args<float>(c, n_sys, (const float2*)x, (float2*)y, c->Dr32.as<float2>(), nullptr, true);
            a.U = reinterpret_cast<float2*>(scratch);
            launch_matvec<float>(L, a, st);
        }
        CK(cudaGetLastError());
        return EELS_OK;
    });
}

extern "C" {

int eels_cl_total(int n, const double* p_eels, const double* p_ext, const double* p_cl, double* out) {
    if (n < 0 || (n > 0 && (!p_eels || !p_ext || !p_cl || !out))) return EELS_E_INVALID_ARG;
    for (int i = 0; i < n; ++i) out[i] = p_eels[i] - p_ext[i] + p_cl[i];
    return EELS_OK;
}

int eels_frank_tamm(double ekin_keV, eels_c128 eps_h, double* dp_dz) {
    if (!dp_dz || !(ekin_keV > 0) || !(eps_h.re > 0) || eps_h.im != 0.0) return EELS_E_INVALID_ARG;
    const double v = electron_speed(ekin_keV);
    const double b2 = v * v * eps_h.re / (kC * kC);   // beta_h^2
    // (2/pi) (dW0/dz) / (hbar^2 w) e with dW0/dz = (mu0/8) e^2 w (1 - 1/beta_h^2), mu0 = 1/(eps0 c^2)
    *dp_dz = b2 <= 1.0 ? 0.0 : kE * kE * (1.0 - 1.0 / b2) / (4.0 * kPi * kEps0 * kC * kC * kHbar * kHbar) * kE;
    return EELS_OK;
}

int eels_vacuum_equivalent(int rule, double ekin_keV, double eps_h, double energy_eV, eels_vacuum_map* out) {
    if (!out || !(ekin_keV > 0) || !(eps_h > 0) || !(energy_eV > 0) ||
        (rule & ~(EELS_SCALE_LENGTH | EELS_SCALE_ULTRAREL)))
        return EELS_E_INVALID_ARG;
    const double m_h = std::sqrt(eps_h), beta_h = electron_speed(ekin_keV) * m_h / kC;
    const double eta = m_h, xi = (rule & EELS_SCALE_LENGTH) ? 1.0 / m_h : 1.0;
    eels_vacuum_map m;
    m.energy_eV = xi * eta * energy_eV;    // omega -> xi eta omega (Eq. 44)
    m.length_scale = 1.0 / xi;             // r -> r / xi (Eq. 43)
    m.eps_p_scale = 1.0 / (eta * eta);     // m_p -> m_p / eta
    m.p_scale = xi;                        // P -> P / xi (Eq. 44), inverted
    if (rule & EELS_SCALE_ULTRAREL) {
        if (!(beta_h > 1.0)) return EELS_E_INVALID_ARG;
        m.ekin_keV = std::numeric_limits<double>::infinity();
        m.p_scale = xi / (beta_h * beta_h);   // Eq. S16: P -> beta_h^2 P at v = c, inverted
    } else {
        if (!(beta_h < 1.0)) return EELS_E_INVALID_ARG;
        // the kinetic energy of speed m_h v (Eq. 47 is its closed form)
        m.ekin_keV = kMeC2keV * (1.0 / std::sqrt((1.0 - beta_h) * (1.0 + beta_h)) - 1.0);
    }
    *out = m;
    return EELS_OK;
}

int eels_extrapolate(int n, const double* d, const double* values, double* value0, double* ci95) {
    if (n < 3 || !d || !values || !value0 || !ci95) return EELS_E_INVALID_ARG;
    // weighted least squares for v(d) = a0 + a1 d + a2 d^2, weights d^-6
    // (errors growing as d^3); 3x3 normal matrix inverted by cofactors
    double m[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, r[3] = {0, 0, 0};
    for (int i = 0; i < n; ++i) {
        if (!(d[i] > 0)) return EELS_E_INVALID_ARG;
        const double wi = 1.0 / std::pow(d[i], 6), b[3] = {1.0, d[i], d[i] * d[i]};
        for (int p = 0; p < 3; ++p) {
            r[p] += wi * b[p] * values[i];
            for (int q = 0; q < 3; ++q) m[p][q] += wi * b[p] * b[q];
        }
    }
    double inv[3][3];
    for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q) {
            const int p1 = (q + 1) % 3, p2 = (q + 2) % 3, q1 = (p + 1) % 3, q2 = (p + 2) % 3;
            inv[p][q] = m[p1][q1] * m[p2][q2] - m[p1][q2] * m[p2][q1];   // cofactor of m[q][p]
        }
    const double det = m[0][0] * inv[0][0] + m[0][1] * inv[1][0] + m[0][2] * inv[2][0];
    if (!(std::fabs(det) > 0)) return EELS_E_INVALID_ARG;
    double a[3];
    for (int p = 0; p < 3; ++p) {
        for (int q = 0; q < 3; ++q) inv[p][q] /= det;
    }
    for (int p = 0; p < 3; ++p) a[p] = inv[p][0] * r[0] + inv[p][1] * r[1] + inv[p][2] * r[2];
    *value0 = a[0];
    *ci95 = 0.0;
    if (n > 3) {
        double chi2 = 0.0;
        for (int i = 0; i < n; ++i) {
            const double e = values[i] - (a[0] + a[1] * d[i] + a[2] * d[i] * d[i]);
            chi2 += e * e / std::pow(d[i], 6);
        }
        *ci95 = 2.0 * std::sqrt(chi2 / (n - 3) * inv[0][0]);
    }
    return EELS_OK;
}

int eels_directions(int n_dir, double* dirs, double* weights) {
    std::vector<double> d, w;
    if (!dirs || !weights || !icosphere(n_dir, d, w)) return EELS_E_INVALID_ARG;
    std::memcpy(dirs, d.data(), d.size() * sizeof(double));
    std::memcpy(weights, w.data(), w.size() * sizeof(double));
    return EELS_OK;
}

}  // extern "C"
