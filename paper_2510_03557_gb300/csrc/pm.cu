// Long-range gravity of the long/short split on a particle mesh (paper
// Sec. IV-A: the long-range part runs in FP64 on a spectral PM solver, the
// short-range part in the particle-particle passes).  With the Gaussian
// split whose short-range factor is S(r) = erfc(r / 2 r_s) +
// r / (sqrt(pi) r_s) exp(-r^2 / 4 r_s^2), the long-range potential is the
// Newtonian one filtered by exp(-k^2 r_s^2), so that the two parts add up to
// Newtonian gravity.  For one periodic box of side L on an ng^3 mesh
// (cell d = L / ng, centres at (i + 1/2) d), all in FP64:
//   1. cloud-in-cell deposit of the mass density (atomic adds),
//   2. forward real FFT (cuFFT),
//   3. phi(k) = -4 pi G rho(k) exp(-k^2 r_s^2) / (k^2 C(k)^2), phi(0) = 0, with
//      C(k) = prod_a sinc^2(k_a d / 2) undoing both cloud-in-cell windows,
//   4. a(k) = -i k phi(k) per axis, zero on that axis's Nyquist plane,
//   5. three inverse FFTs and the cloud-in-cell gather at every particle.
// The atomic deposit sums in no fixed order: results agree to rounding.
#include "sim.h"

#include <cufft.h>

namespace crk {

namespace {

constexpr int kT = 256;
constexpr double kPi = 3.14159265358979323846;

inline unsigned nblocks(int64_t n) { return (unsigned)((n + kT - 1) / kT); }

// The 8 cells and weights of particle coordinate x along one axis:
// lower cell index i0 (mod ng) and the fraction f towards the next centre.
__device__ __forceinline__ void cic_axis(double x, double d, int ng, int &i0, double &f)
{
    const double s = x / d - 0.5;
    const double fl = floor(s);
    f = s - fl;
    int i = (int)fl % ng;
    if (i < 0) i += ng;
    i0 = i;
}

__global__ void pm_deposit_k(State s, int64_t n, double L, int ng, double *rho)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double d = L / ng;
    const double inv_d3 = 1.0 / (d * d * d);
    int ix, iy, iz;
    double fx, fy, fz;
    cic_axis(s.x[k], d, ng, ix, fx);
    cic_axis(s.y[k], d, ng, iy, fy);
    cic_axis(s.z[k], d, ng, iz, fz);
    const double m = s.m[k];
#pragma unroll
    for (int ox = 0; ox < 2; ++ox) {
        const double wx = ox ? fx : 1.0 - fx;
        const int cx = (ix + ox) % ng;
#pragma unroll
        for (int oy = 0; oy < 2; ++oy) {
            const double wy = oy ? fy : 1.0 - fy;
            const int cy = (iy + oy) % ng;
#pragma unroll
            for (int oz = 0; oz < 2; ++oz) {
                const double wz = oz ? fz : 1.0 - fz;
                const int cz = (iz + oz) % ng;
                atomicAdd(&rho[((int64_t)cx * ng + cy) * ng + cz], m * (wx * wy * wz) * inv_d3);
            }
        }
    }
}

__device__ __forceinline__ double sinc(double x) { return x == 0.0 ? 1.0 : sin(x) / x; }

// Mode (ix, iy, iz) of the half-complex layout (last axis ng/2 + 1); the
// inverse transforms are unnormalised, so 1/ng^3 is folded in here.
__global__ void pm_green_k(const double2 *rk, int ng, double L, double G, double rs, double2 *ax,
                           double2 *ay, double2 *az)
{
    const int nz = ng / 2 + 1;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)ng * ng * nz) return;
    const int iz = (int)(t % nz);
    const int iy = (int)((t / nz) % ng);
    const int ix = (int)(t / ((int64_t)nz * ng));
    const int fx = ix < ng / 2 ? ix : ix - ng, fy = iy < ng / 2 ? iy : iy - ng, fz = iz;
    const double kf = 2.0 * kPi / L;
    const double kx = kf * fx, ky = kf * fy, kz = kf * fz;
    const double k2 = kx * kx + ky * ky + kz * kz;
    double2 zero;
    zero.x = 0.0;
    zero.y = 0.0;
    if (k2 == 0.0) {
        ax[t] = zero;
        ay[t] = zero;
        az[t] = zero;
        return;
    }
    const double d = L / ng;
    const double c = sinc(0.5 * kx * d) * sinc(0.5 * ky * d) * sinc(0.5 * kz * d);
    const double C = c * c;
    const double fac = -4.0 * kPi * G * exp(-k2 * rs * rs) / (k2 * C * C) / ((double)ng * ng * ng);
    const double2 r = rk[t];
    const double px = r.x * fac, py = r.y * fac;
    // -i k phi = (k phi_im, -k phi_re); no derivative on the Nyquist plane
    const double kxd = (ix == ng / 2) ? 0.0 : kx, kyd = (iy == ng / 2) ? 0.0 : ky,
                 kzd = (iz == ng / 2) ? 0.0 : kz;
    double2 o;
    o.x = kxd * py; o.y = -kxd * px; ax[t] = o;
    o.x = kyd * py; o.y = -kyd * px; ay[t] = o;
    o.x = kzd * py; o.y = -kzd * px; az[t] = o;
}

// Gather of the three mesh fields at every particle; written at the
// particle's sorted index, or at its load-order index when load_order.
__global__ void pm_interp_k(State s, int64_t n, double L, int ng, const double *gx, const double *gy,
                            const double *gz, double *acc, int load_order)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double d = L / ng;
    int ix, iy, iz;
    double fx, fy, fz;
    cic_axis(s.x[k], d, ng, ix, fx);
    cic_axis(s.y[k], d, ng, iy, fy);
    cic_axis(s.z[k], d, ng, iz, fz);
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
#pragma unroll
    for (int ox = 0; ox < 2; ++ox) {
        const double wx = ox ? fx : 1.0 - fx;
        const int cx = (ix + ox) % ng;
#pragma unroll
        for (int oy = 0; oy < 2; ++oy) {
            const double wy = oy ? fy : 1.0 - fy;
            const int cy = (iy + oy) % ng;
#pragma unroll
            for (int oz = 0; oz < 2; ++oz) {
                const double wz = oz ? fz : 1.0 - fz;
                const int cz = (iz + oz) % ng;
                const int64_t c = ((int64_t)cx * ng + cy) * ng + cz;
                const double w = wx * wy * wz;
                a0 += gx[c] * w;
                a1 += gy[c] * w;
                a2 += gz[c] * w;
            }
        }
    }
    const int64_t o = load_order ? (int64_t)s.id[k] : k;
    acc[3 * o] = a0;
    acc[3 * o + 1] = a1;
    acc[3 * o + 2] = a2;
}

const char *cufft_msg(cufftResult r)
{
    switch (r) {
    case CUFFT_SUCCESS: return "success";
    case CUFFT_ALLOC_FAILED: return "allocation failed";
    case CUFFT_INVALID_VALUE: return "invalid value";
    case CUFFT_EXEC_FAILED: return "execution failed";
    default: return "cuFFT error";
    }
}

}  // namespace

#define CUFFT_CK(call)                                                                          \
    do {                                                                                        \
        cufftResult r_ = (call);                                                                \
        if (r_ != CUFFT_SUCCESS)                                                                \
            return fail(r_ == CUFFT_ALLOC_FAILED ? CRK_ENOMEM : CRK_ECUDA, "%s failed: %s", #call, \
                        cufft_msg(r_));                                                         \
    } while (0)

int pm_accelerations(crk_sim *s, double *acc, bool load_order)
{
    const int ng = s->prm.pm_grid;
    const BoxDev &bx = s->boxes[0];
    const int64_t n = s->n;
    cudaStream_t st = s->st;
    const size_t cells = (size_t)ng * ng * ng, modes = (size_t)ng * ng * (ng / 2 + 1);
    if (s->pm_ng != ng) {
        if (s->pm_ng > 0) {
            cufftDestroy((cufftHandle)s->pm_fwd);
            cufftDestroy((cufftHandle)s->pm_inv);
            s->pm_ng = 0;
        }
        cufftHandle f, i;
        CUFFT_CK(cufftPlan3d(&f, ng, ng, ng, CUFFT_D2Z));
        cufftResult r = cufftPlan3d(&i, ng, ng, ng, CUFFT_Z2D);
        if (r != CUFFT_SUCCESS) {
            cufftDestroy(f);
            return fail(CRK_ECUDA, "cufftPlan3d failed: %s", cufft_msg(r));
        }
        s->pm_fwd = (int)f;
        s->pm_inv = (int)i;
        s->pm_ng = ng;
    }
    RET(s->pm_mesh.ensure(cells * 4 * sizeof(double)));
    RET(s->pm_modes.ensure(modes * 4 * sizeof(double2)));
    double *rho = s->pm_mesh.as<double>();
    double *g[3] = {rho + cells, rho + 2 * cells, rho + 3 * cells};
    double2 *rk = s->pm_modes.as<double2>();
    double2 *ck[3] = {rk + modes, rk + 2 * modes, rk + 3 * modes};
    CUFFT_CK(cufftSetStream((cufftHandle)s->pm_fwd, st));
    CUFFT_CK(cufftSetStream((cufftHandle)s->pm_inv, st));
    CK(cudaMemsetAsync(rho, 0, cells * sizeof(double), st));
    if (n > 0) pm_deposit_k<<<nblocks(n), kT, 0, st>>>(s->sa, n, bx.L, ng, rho);
    CUFFT_CK(cufftExecD2Z((cufftHandle)s->pm_fwd, rho, reinterpret_cast<cufftDoubleComplex *>(rk)));
    pm_green_k<<<nblocks((int64_t)modes), kT, 0, st>>>(rk, ng, bx.L, bx.G, bx.r_split, ck[0], ck[1], ck[2]);
    for (int a = 0; a < 3; ++a)
        CUFFT_CK(cufftExecZ2D((cufftHandle)s->pm_inv, reinterpret_cast<cufftDoubleComplex *>(ck[a]), g[a]));
    if (n > 0) pm_interp_k<<<nblocks(n), kT, 0, st>>>(s->sa, n, bx.L, ng, g[0], g[1], g[2], acc,
                                               load_order ? 1 : 0);
    note_launches(3 + 4);
    CK(cudaGetLastError());
    return CRK_OK;
}

void pm_release(crk_sim *s)
{
    if (s->pm_ng > 0) {
        cufftDestroy((cufftHandle)s->pm_fwd);
        cufftDestroy((cufftHandle)s->pm_inv);
        s->pm_ng = 0;
    }
    s->pm_mesh.release();
    s->pm_modes.release();
}

}  // namespace crk
