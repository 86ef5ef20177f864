// Internal launch interface between the host engine and the CUDA kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <array>
#include <vector>

#include "common.cuh"
#include "fft.cuh"

namespace eels {

// Process-wide count of kernels this library has launched (graph replays
// add their kernel nodes; launches recorded during a stream capture are not
// counted until the graph runs).
extern std::atomic<long long> g_kernel_launches;
extern thread_local bool g_capturing;
inline void count_launch(int n = 1) {
    if (!g_capturing) g_kernel_launches += n;
}

// Lattice description shared by every kernel (device pointers).
struct LatticeDev {
    int Nx, Ny, Nz, N;            // box extents, occupied cells
    int Mx, My, Mz;               // padded FFT extents (even)
    int Hx, Hy, Hz;               // reduced D-hat extents: M/2 + 1
    const int* cellmap;           // [Nx][Ny][Nz] (slab-major) -> internal dipole index or -1
    const uint8_t* mat;           // [N] 0-based material
    const int* dip_cell;          // [N] internal dipole -> cell index ix + Nx (iy + Ny iz)
    const int2* col_range;        // [Ny][Nx] occupied iz range [first, last+1) (first = last = 0 if empty)
    const int4* colinfo;          // [Nx][Ny] (index of the column's first dipole - first, first, last+1, 0)
    int contig;                   // 1 if every column's occupied cells are contiguous in z (colinfo is exact)
    int nmat;                     // materials used by the lattice (1: one coefficient per system)
    const double* igt;            // D-hat build only: cell tables of the igt_so interaction (igt.cu), or
                                  // nullptr for point dipoles
    FftPlan px, py, pz;
    int xw32, xw64;               // x-pass tile width chosen by the autotuner (0: size heuristic)
    int xmode;                    // register x pass: 0 choose by availability, 1 direct loads, 2 tensor copies
    const double2* tw64x; const double2* tw64y; const double2* tw64z;   // exp(-2 pi i t / M)
    const float2* tw32x; const float2* tw32y; const float2* tw32z;
};

// y = diag[m] x - coef[m] * conv(coef[m'] x) / M for a batch of systems.
// conv(u)_i = sum_{j != i} G~'(r_i - r_j) u_j evaluated by zero-padded FFT.
// Per-system per-material coefficients are FP64 [S][EELS_MAX_MAT].
template <typename Rl>
struct MatvecArgs {
    const cx<Rl>* x;              // [S][3][N]
    cx<Rl>* y;                    // [S][3][N]
    cx<Rl>* U;                    // scratch [S][3][My][Nx][Mz]
    const cx<Rl>* Dr;             // reduced D-hat [slot][6][Hy][Hx][Hz]
    const int* sys_slot;          // [S] D-hat slot of each system
    const double2* coef;          // [S][EELS_MAX_MAT]
    const double2* diag;          // [S][EELS_MAX_MAT]
    const int* active;            // [S] or nullptr
    double* dot_part;             // optional [S][3 Nx][4]: per-slab sum x.y (unconjugated), written by the
                                  // three-pass path's last kernel
    const float2* Dx;             // FP32 D-hat [slot][Hy][Hz][6][Hx] (register x pass), or nullptr
    int S;
    int spb;                      // systems per x-pass block (consecutive systems that usually share a
                                  // D-hat slot: the beams of one energy); 0 or 1: one
};

// Cell-integrated Green's tensor (igt_so): lattice offsets of max-norm <=
// IGT_NEAR take exp(i kappa R) (-T0 + i kappa T1 + kappa^2 T2); the host
// table holds, per offset (x fastest over [-IGT_NEAR, IGT_NEAR]^3), T0, T1,
// T2 in the component order xx xy xz yy yz zz (18 doubles), lattice units.
constexpr int IGT_NEAR = 3;
constexpr double IGT_C1 = 2.3800773639795505;   // integral of 1/|u| over the unit cube: 3 ln(2 + sqrt 3) - pi/2
const std::vector<double>& igt_tables();

// Returns true when a.dot_part was filled (three-pass path).
template <typename Rl>
bool launch_matvec(const LatticeDev& L, const MatvecArgs<Rl>& a, cudaStream_t st);

// D-hat build for n_slot energies: kappa[slot] = k d (complex).  G scratch
// [n_slot][6][My][Mx][Mz] FP64; outputs reduced D-hat FP64 and FP32.
void launch_dhat_build(const LatticeDev& L, int n_slot, const double2* kappa, double2* Gscratch,
                       double2* Dr64, float2* Dr32, cudaStream_t st, float2* Dx32 = nullptr);
// FP32 copy Dx[slot][ky][kz][comp][kx] of the octant D-hat (read by the
// register-resident x pass).
void launch_dhat_interleave(const LatticeDev& L, int n_slot, const double2* Dr64, float2* Dx, cudaStream_t st);
// Register-resident x pass (Mx = 64 or 128, FP32): false when the lattice or
// the arguments do not suit it (the caller then launches the shared-memory one).
bool xpass_reg_supported(const LatticeDev& L);
bool launch_xpass_reg(const LatticeDev& L, const MatvecArgs<float>& a, cudaStream_t st);
// Times the register x pass on the systems of a (CUDA events on st; not
// during a stream capture) for each way of moving U (direct loads, tensor
// copies when available) and each number of systems per block in
// {1, 2, 4, 8, 16} up to max_spb, and returns the fastest in *mode, *spb.
// The x pass transforms a.U in place: its contents are lost.  *log
// receives every timed candidate as (mode, spb, ms of three launches).
void autotune_xreg(const LatticeDev& L, const MatvecArgs<float>& a, int max_spb, cudaStream_t st, int* mode, int* spb,
                   std::vector<std::array<float, 3>>* log);

// Bounded device-side waits that gave up since the library was loaded (each
// one left its kernel's results incomplete).  Reading it synchronises the device.
unsigned int wait_timeouts();

size_t matvec_smem_bytes(const LatticeDev& L, bool fp64);
// Times the x pass with every tile width whose shared memory fits, on the
// systems of a (CUDA events on st; not during a stream capture), and returns
// the fastest width.  The x pass transforms a.U in place: its contents are
// lost.
template <typename Rl>
int autotune_xpass(const LatticeDev& L, const MatvecArgs<Rl>& a, cudaStream_t st);
int matvec_passes(const LatticeDev& L, bool fp64);   // 3 (fused slabs) or 5

// Raise the dynamic shared-memory limit of every kernel instance (call once
// per device before any launch or stream capture).
void prepare_kernels();

// Incident field for S systems (per-system params in SysField), FP64 out [S][3][N].
struct SysField {
    double2 kt;         // omega d / (gamma_h v): Bessel argument per unit b/d
    double2 inv_gamma;  // 1 / gamma_h
    double2 pref_unit;  // phase of the Eq. 25 prefactor
    double wdv;         // omega d / v
    double x0, y0;      // beam, lattice units relative to the lattice centre (electron along +z)
    // electron along an arbitrary direction n: the trajectory passes through p
    // (lattice units relative to the lattice centre); along_z selects the +z
    // kernels, for which p = (x0, y0, 0) and n = z
    double px, py, pz, nx, ny, nz;
    int along_z;
};
// along_z: every system's electron moves along +z (the per-column kernel)
void launch_incident_field(const LatticeDev& L, int S, const SysField* sys, bool along_z, double2* e,
                           cudaStream_t st);
void launch_aux_field(const LatticeDev& L, int S, const SysField* sys, const double2* e, double2* ea, cudaStream_t st);
void launch_bessel(const double2* z, double2* k0, double2* k1, int n, cudaStream_t st);

}  // namespace eels
