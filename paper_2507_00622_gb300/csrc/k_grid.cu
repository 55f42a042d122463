// k_grid.cu -- initial-condition generators and the LD-indicator stencil.
#include <math.h>

#include "chs_internal.cuh"

namespace chs {

// Henon-Heiles section grid (Eq. Ham_HH at x = 0):
//   p_x^2 = 2E - p_y^2 - y^2 + 2 y^3 / 3.
// Every operation is an explicitly rounded IEEE double operation in the order
// written, so the FORBIDDEN decision (sign of the radicand) is reproducible
// bit for bit by any IEEE implementation that evaluates the same expression.
__global__ void k_grid_ics(const double E, const double y0, const double y1, const int ny,
                           const double py0, const double py1, const int npy,
                           double* __restrict__ ics, int32_t* __restrict__ status)
{
    const int64_t n = (int64_t)ny * npy;
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n) return;
    const int iy = (int)(o / npy), ip = (int)(o % npy);
    const double dy = __ddiv_rn(__dsub_rn(y1, y0), (double)ny);
    const double dpy = __ddiv_rn(__dsub_rn(py1, py0), (double)npy);
    const double y = __dadd_rn(y0, __dmul_rn(__dadd_rn((double)iy, 0.5), dy));
    const double py = __dadd_rn(py0, __dmul_rn(__dadd_rn((double)ip, 0.5), dpy));
    const double cubic = __ddiv_rn(__dmul_rn(__dmul_rn(__dmul_rn(2.0, y), y), y), 3.0);
    const double rad = __dadd_rn(__dsub_rn(__dsub_rn(__dmul_rn(2.0, E), __dmul_rn(py, py)),
                                           __dmul_rn(y, y)),
                                 cubic);
    if (rad < 0.0) {
        const double qnan = __longlong_as_double(0x7ff8000000000000LL);
        status[o] = CHS_ORBIT_FORBIDDEN;
        ics[0 * n + o] = qnan;
        ics[1 * n + o] = qnan;
        ics[2 * n + o] = qnan;
        ics[3 * n + o] = qnan;
    } else {
        status[o] = CHS_ORBIT_OK;
        ics[0 * n + o] = 0.0;
        ics[1 * n + o] = y;
        ics[2 * n + o] = __dsqrt_rn(rad);
        ics[3 * n + o] = py;
    }
}

cudaError_t launch_grid_ics(double E, double y0, double y1, int ny, double py0, double py1, int npy,
                            double* ics, int32_t* status, cudaStream_t st)
{
    const int64_t n = (int64_t)ny * npy;
    if (n == 0) return cudaSuccess;
    k_grid_ics<<<blocks_for(n, 256), 256, 0, st>>>(E, y0, y1, ny, py0, py1, npy, ics, status);
    return cudaGetLastError();
}

// LD-based indicators on the section grid (o = iy * npy + ipy), two grid
// directions, one-cell offset:
//   D_L = (|LD(y+) - LD(y-)| / LD + |LD(p+) - LD(p-)| / LD) / 4
//   S_L = (|2 - (LD(y+) + LD(y-)) / LD| + |2 - (LD(p+) + LD(p-)) / LD|) / 2
// NaN on the border and next to any cell whose status is not OK.  Explicitly
// rounded, uncontracted operations in the order written.
__global__ void k_ld_stencil(const int ny, const int npy, const double* __restrict__ ld,
                             const int32_t* __restrict__ status, double* __restrict__ out)
{
    const int64_t n = (int64_t)ny * npy;
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n) return;
    const int iy = (int)(o / npy), ip = (int)(o % npy);
    const double qnan = __longlong_as_double(0x7ff8000000000000LL);
    double dl = qnan, sl = qnan;
    if (iy > 0 && iy < ny - 1 && ip > 0 && ip < npy - 1) {
        const bool ok = status[o] == CHS_ORBIT_OK && status[o - npy] == CHS_ORBIT_OK &&
                        status[o + npy] == CHS_ORBIT_OK && status[o - 1] == CHS_ORBIT_OK &&
                        status[o + 1] == CHS_ORBIT_OK;
        if (ok) {
            const double c = ld[o];
            const double ym = ld[o - npy], yp = ld[o + npy], pm = ld[o - 1], pp = ld[o + 1];
            const double dsum = __dadd_rn(__ddiv_rn(fabs(__dsub_rn(yp, ym)), c),
                                          __ddiv_rn(fabs(__dsub_rn(pp, pm)), c));
            const double ssum = __dadd_rn(fabs(__dsub_rn(2.0, __ddiv_rn(__dadd_rn(yp, ym), c))),
                                          fabs(__dsub_rn(2.0, __ddiv_rn(__dadd_rn(pp, pm), c))));
            dl = __ddiv_rn(dsum, 4.0);
            sl = __ddiv_rn(ssum, 2.0);
        }
    }
    out[o] = dl;
    out[n + o] = sl;
}

cudaError_t launch_ld_stencil(int ny, int npy, const double* ld, const int32_t* status, double* out,
                              cudaStream_t st)
{
    const int64_t n = (int64_t)ny * npy;
    if (n == 0) return cudaSuccess;
    k_ld_stencil<<<blocks_for(n, 256), 256, 0, st>>>(ny, npy, ld, status, out);
    return cudaGetLastError();
}

// FPUT initial conditions from normal-mode amplitudes (FPU example of Sec.
// Examples): q_i = sqrt(2/(N+1)) sum_m Q_m sin(i m pi/(N+1)), p likewise,
// then the state is scaled onto H = E with s^2 = 2E / (H2 + sqrt(H2^2 + 4 H4 E))
// (alpha = 0: H(s x) = s^2 H2 + s^4 H4).  One orbit per thread; the state is
// written straight to its SoA slots.
__global__ void k_fput_mode_ics(const SysPar sp, const int64_t n, const double* __restrict__ Qm,
                                const double* __restrict__ Pm, const double* __restrict__ E,
                                double* __restrict__ ics)
{
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n) return;
    const int N = sp.n_dof;
    const double pi = 3.141592653589793;
    const double nrm = sqrt(2.0 / (double)(N + 1));
    double H2 = 0.0, H4 = 0.0, qprev = 0.0;
    for (int i = 1; i <= N; ++i) {
        double aq = 0.0, ap = 0.0;
        for (int m = 1; m <= N; ++m) {
            const double sn = sin((double)i * (double)m * pi / (double)(N + 1));
            aq = fma(Qm[(int64_t)(m - 1) * n + o], sn, aq);
            ap = fma(Pm[(int64_t)(m - 1) * n + o], sn, ap);
        }
        const double q = nrm * aq, p = nrm * ap;
        ics[(int64_t)(i - 1) * n + o] = q;
        ics[(int64_t)(N + i - 1) * n + o] = p;
        const double r = q - qprev;
        H2 += 0.5 * p * p + 0.5 * sp.kk * r * r;
        H4 += 0.25 * sp.beta * r * r * r * r;
        qprev = q;
    }
    H2 += 0.5 * sp.kk * qprev * qprev;  // bond N+1 to the fixed end
    H4 += 0.25 * sp.beta * qprev * qprev * qprev * qprev;
    const double Eo = E[o];
    const double sc = sqrt(2.0 * Eo / (H2 + sqrt(H2 * H2 + 4.0 * H4 * Eo)));
    for (int c = 0; c < 2 * N; ++c) ics[(int64_t)c * n + o] *= sc;
}

cudaError_t launch_fput_mode_ics(const SysPar& sp, int64_t n, const double* Qm, const double* Pm,
                                 const double* E, double* ics, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    k_fput_mode_ics<<<blocks_for(n, 128), 128, 0, st>>>(sp, n, Qm, Pm, E, ics);
    return cudaGetLastError();
}

// Quartic-3 initial conditions on energy shells: u = dir / |dir|, scaled by s
// with H(s u) = E, s^2 = 2E / (H2 + sqrt(H2^2 + 4 H4 E)), H2 = |u|^2 / 2,
// H4 = eps (u1^2 u2^2 + u2^2 u3^2 + u1^2 u3^2).
__global__ void k_shell_ics(const SysPar sp, const int64_t n, const double* __restrict__ dirs,
                            const double* __restrict__ E, double* __restrict__ ics)
{
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n) return;
    double u[6], nr = 0.0;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        u[c] = dirs[c * n + o];
        nr = fma(u[c], u[c], nr);
    }
    const double inv = 1.0 / sqrt(nr);
    double H2 = 0.0;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        u[c] *= inv;
        H2 = fma(0.5 * u[c], u[c], H2);
    }
    const double a = u[0] * u[0], b = u[1] * u[1], c2 = u[2] * u[2];
    const double H4 = sp.eps * (a * b + b * c2 + a * c2);
    const double Eo = E[o];
    const double sc = sqrt(2.0 * Eo / (H2 + sqrt(H2 * H2 + 4.0 * H4 * Eo)));
#pragma unroll
    for (int c = 0; c < 6; ++c) ics[c * n + o] = sc * u[c];
}

cudaError_t launch_shell_ics(const SysPar& sp, int64_t n, const double* dirs, const double* E,
                             double* ics, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    k_shell_ics<<<blocks_for(n, 128), 128, 0, st>>>(sp, n, dirs, E, ics);
    return cudaGetLastError();
}

}  // namespace chs
