// Fast-electron incident field at the dipoles (Eq. 25 of the paper), FP64.
//
// E_inc(r) = P exp(i w (z - z0)/v) ((x-x0)/b K1(a), (y-y0)/b K1(a), -(i/gamma_h) K0(a)),
// a = w b / (gamma_h v), P = q w / (2 pi eps0 m_h^2 v^2 gamma_h).
// The kernel writes E_inc / |P| in lattice units: b and z in units of d,
// so a = kt * b' with kt = w d / (gamma_h v) and the phase is wdv * z'.
// K0/K1 depend on the column (ix, iy) only, so one thread evaluates them
// once per column and sweeps the occupied cells of that column.
#include "bessel.cuh"
#include "kernels.h"

namespace eels {

__global__ void k_bessel(const double2* z, double2* k0, double2* k1, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 a, b;
    bessel_k01(z[i], &a, &b);
    k0[i] = a;
    k1[i] = b;
}

__global__ void k_einc(LatticeDev L, const SysField* sys, double2* e) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= L.Nx * L.Ny) return;
    const int s = blockIdx.y;
    const int2 rg = L.col_range[col];
    if (rg.x >= rg.y) return;
    const int ix = col % L.Nx, iy = col / L.Nx;
    const SysField p = sys[s];
    const double xr = (ix + 0.5) - 0.5 * L.Nx - p.x0;
    const double yr = (iy + 0.5) - 0.5 * L.Ny - p.y0;
    const double b = hypot(xr, yr);
    double2 K0, K1;
    bessel_k01(b * p.kt, &K0, &K1);
    const double2 txy = (1.0 / b) * (p.pref_unit * K1);
    const double2 ex = xr * txy, ey = yr * txy;
    const double2 ez = p.pref_unit * (make_double2(p.inv_gamma.y, -p.inv_gamma.x) * K0);   // -i / gamma_h
    const size_t N = (size_t)L.N;
    double2* e0 = e + (size_t)s * 3 * N;
    for (int iz = rg.x; iz < rg.y; ++iz) {
        const int dip = L.cellmap[((size_t)ix * L.Ny + iy) * L.Nz + iz];
        if (dip < 0) continue;
        const double zr = (iz + 0.5) - 0.5 * L.Nz;
        double sn, cs;
        sincos(p.wdv * zr, &sn, &cs);
        const double2 ph = make_double2(cs, sn);
        e0[dip] = ex * ph;
        e0[N + dip] = ey * ph;
        e0[2 * N + dip] = ez * ph;
    }
}

// Electron along an arbitrary direction n through p: per dipole, with
// r' = r - p, z' = r'.n and the transverse vector b = r' - z' n,
//   E_inc = P exp(i w z'/v) (b/|b| K1(a) - (i/gamma_h) K0(a) n),  a = w |b| / (gamma_h v),
// Eq. 25 written in the electron's frame.  One thread per dipole (K0/K1 are
// no longer shared along a lattice column).
__global__ void k_einc_dir(LatticeDev L, const SysField* sys, double2* e) {
    const int s = blockIdx.y;
    const SysField p = sys[s];
    const size_t N = (size_t)L.N;
    double2* e0 = e + (size_t)s * 3 * N;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L.N; i += gridDim.x * blockDim.x) {
        const int cell = L.dip_cell[i];
        const int ix = cell % L.Nx, iy = (cell / L.Nx) % L.Ny, iz = cell / (L.Nx * L.Ny);
        const double rx = (ix + 0.5) - 0.5 * L.Nx - p.px;
        const double ry = (iy + 0.5) - 0.5 * L.Ny - p.py;
        const double rz = (iz + 0.5) - 0.5 * L.Nz - p.pz;
        const double zp = rx * p.nx + ry * p.ny + rz * p.nz;
        const double bx = rx - zp * p.nx, by = ry - zp * p.ny, bz = rz - zp * p.nz;
        const double b = sqrt(bx * bx + by * by + bz * bz);
        double2 K0, K1;
        bessel_k01(b * p.kt, &K0, &K1);
        double sn, cs;
        sincos(p.wdv * zp, &sn, &cs);
        const double2 ph = make_double2(cs, sn);
        const double2 t = (1.0 / b) * (ph * (p.pref_unit * K1));
        const double2 l = ph * (p.pref_unit * (make_double2(p.inv_gamma.y, -p.inv_gamma.x) * K0));   // -i / gamma_h
        e0[i] = bx * t + p.nx * l;
        e0[N + i] = by * t + p.ny * l;
        e0[2 * N + i] = bz * t + p.nz * l;
    }
}

// E_a = (-E_x, -E_y, E_z) exp(-2 i w (z - z0)/v)   (Eq. 34, second form); for
// an arbitrary direction, (-E + 2 (E.n) n) exp(-2 i w z'/v)
__global__ void k_eaux(LatticeDev L, const SysField* sys, const double2* e, double2* ea) {
    const int s = blockIdx.y;
    const size_t N = (size_t)L.N, off = (size_t)s * 3 * N;
    const double w = sys[s].wdv;
    if (!sys[s].along_z) {
        const SysField p = sys[s];
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L.N; i += gridDim.x * blockDim.x) {
            const int cell = L.dip_cell[i];
            const int ix = cell % L.Nx, iy = (cell / L.Nx) % L.Ny, iz = cell / (L.Nx * L.Ny);
            const double zp = ((ix + 0.5) - 0.5 * L.Nx - p.px) * p.nx + ((iy + 0.5) - 0.5 * L.Ny - p.py) * p.ny +
                              ((iz + 0.5) - 0.5 * L.Nz - p.pz) * p.nz;
            double sn, cs;
            sincos(-2.0 * w * zp, &sn, &cs);
            const double2 ph = make_double2(cs, sn);
            const double2 ex = e[off + i], ey = e[off + N + i], ez = e[off + 2 * N + i];
            const double2 en2 = 2.0 * (p.nx * ex + p.ny * ey + p.nz * ez);
            ea[off + i] = ph * (p.nx * en2 - ex);
            ea[off + N + i] = ph * (p.ny * en2 - ey);
            ea[off + 2 * N + i] = ph * (p.nz * en2 - ez);
        }
        return;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L.N; i += gridDim.x * blockDim.x) {
        const int iz = L.dip_cell[i] / (L.Nx * L.Ny);
        const double zr = (iz + 0.5) - 0.5 * L.Nz;
        double sn, cs;
        sincos(-2.0 * w * zr, &sn, &cs);
        const double2 ph = make_double2(cs, sn);
        ea[off + i] = -(ph * e[off + i]);
        ea[off + N + i] = -(ph * e[off + N + i]);
        ea[off + 2 * N + i] = ph * e[off + 2 * N + i];
    }
}

void launch_aux_field(const LatticeDev& L, int S, const SysField* sys, const double2* e, double2* ea, cudaStream_t st) {
    count_launch();
    k_eaux<<<dim3((L.N + 255) / 256, S), 256, 0, st>>>(L, sys, e, ea);
}

void launch_bessel(const double2* z, double2* k0, double2* k1, int n, cudaStream_t st) {
    if (n <= 0) return;
    count_launch();
    k_bessel<<<(n + 127) / 128, 128, 0, st>>>(z, k0, k1, n);
}

void launch_incident_field(const LatticeDev& L, int S, const SysField* sys, bool along_z, double2* e,
                           cudaStream_t st) {
    count_launch();
    if (along_z) {
        const int cols = L.Nx * L.Ny;
        k_einc<<<dim3((cols + 127) / 128, S), 128, 0, st>>>(L, sys, e);
    } else {
        k_einc_dir<<<dim3((L.N + 127) / 128, S), 128, 0, st>>>(L, sys, e);
    }
}

}  // namespace eels
