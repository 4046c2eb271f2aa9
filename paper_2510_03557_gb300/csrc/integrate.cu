// Fixed-step kick-drift-kick on the FP64 master state, FP64 global sums and
// the scatter of results back to the caller's particle order.  All flat,
// memory-bound kernels (coalesced SoA reads; the order-restoring scatter is
// the only uncoalesced access).
#include "crk_internal.h"

namespace crk {

namespace {

constexpr int kT = 256;

inline unsigned nblocks(int64_t n) { return (unsigned)((n + kT - 1) / kT); }

// x + dt v wrapped into [0, L); a value that rounds up to L maps to 0.
__device__ __forceinline__ double drift_wrap(double x, double dt, double v, double L)
{
    double y = __dadd_rn(x, __dmul_rn(dt, v));
    if (y >= L) y -= L;
    if (y < 0.0) {
        y += L;
        if (y >= L) y = 0.0;
    }
    return y;
}

// First half kick and drift:  v += dt/2 a;  u += dt/2 du (gas, floored);
// x = wrap(x + dt v).  Products and sums rounded separately.
__global__ void kick_drift_k(State s, const BoxDev *__restrict__ boxes, int64_t n,
                             unsigned long long *nfloor)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const BoxDev &bx = boxes[s.slot[k]];
    const double hdt = bx.hdt, dt = bx.dt, L = bx.L;
    const double vx = __dadd_rn(s.vx[k], __dmul_rn(hdt, s.ax[k]));
    const double vy = __dadd_rn(s.vy[k], __dmul_rn(hdt, s.ay[k]));
    const double vz = __dadd_rn(s.vz[k], __dmul_rn(hdt, s.az[k]));
    s.vx[k] = vx;
    s.vy[k] = vy;
    s.vz[k] = vz;
    if (s.species[k] == CRK_GAS) {
        double u = __dadd_rn(s.u[k], __dmul_rn(hdt, s.du[k]));
        if (u < bx.u_floor) {
            u = bx.u_floor;
            atomicAdd(nfloor, 1ull);
        }
        s.u[k] = u;
    }
    s.x[k] = drift_wrap(s.x[k], dt, vx, L);
    s.y[k] = drift_wrap(s.y[k], dt, vy, L);
    s.z[k] = drift_wrap(s.z[k], dt, vz, L);
}

// Second half kick with the new rates; the new rates become a_old, du_old.
template <typename R>
__global__ void final_kick_k(PassArgs a, unsigned long long *nfloor)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.n) return;
    const BoxDev &bx = a.boxes[a.s.slot[k]];
    const double hdt = bx.hdt;
    const Vec4<R> g = reinterpret_cast<const Vec4<R> *>(a.acc_g)[k];
    double ax, ay, az, du = 0.0;
    const bool gas = a.s.species[k] == CRK_GAS;
    if (gas) {
        const Vec4<R> hh = reinterpret_cast<const Vec4<R> *>(a.acc_h)[k];
        ax = (double)hh.x + (double)g.x;
        ay = (double)hh.y + (double)g.y;
        az = (double)hh.z + (double)g.z;
        du = (double)hh.w;
    } else {
        ax = (double)g.x;
        ay = (double)g.y;
        az = (double)g.z;
    }
    if (a.acc_pm) {
        ax = __dadd_rn(ax, a.acc_pm[3 * k]);
        ay = __dadd_rn(ay, a.acc_pm[3 * k + 1]);
        az = __dadd_rn(az, a.acc_pm[3 * k + 2]);
    }
    a.s.vx[k] = __dadd_rn(a.s.vx[k], __dmul_rn(hdt, ax));
    a.s.vy[k] = __dadd_rn(a.s.vy[k], __dmul_rn(hdt, ay));
    a.s.vz[k] = __dadd_rn(a.s.vz[k], __dmul_rn(hdt, az));
    if (gas) {
        double u = __dadd_rn(a.s.u[k], __dmul_rn(hdt, du));
        if (u < bx.u_floor) {
            u = bx.u_floor;
            atomicAdd(nfloor, 1ull);
        }
        a.s.u[k] = u;
    }
    a.s.ax[k] = ax;
    a.s.ay[k] = ay;
    a.s.az[k] = az;
    a.s.du[k] = du;
}

// Block partial sums of 4 FP64 quantities, then one block adds the partials
// in a fixed order (deterministic).
__device__ void block_sum4(double v[4], double *dst)
{
    __shared__ double sh[4][kT / 32];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_xor_sync(0xffffffffu, v[c], o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < 4; ++c) sh[c][w] = v[c];
    __syncthreads();
    if (threadIdx.x < 4) {
        double s = 0.0;
        for (int q = 0; q < kT / 32; ++q) s += sh[threadIdx.x][q];
        dst[threadIdx.x] = s;
    }
}

template <typename R>
__global__ void rate_sums_k(PassArgs a, double *partial)
{
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < a.n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const double m = a.s.m[k];
        const Vec4<R> g = reinterpret_cast<const Vec4<R> *>(a.acc_g)[k];
        double ax = g.x, ay = g.y, az = g.z;
        if (a.s.species[k] == CRK_GAS) {
            const Vec4<R> hh = reinterpret_cast<const Vec4<R> *>(a.acc_h)[k];
            const Vec4<R> r1 = reinterpret_cast<const Vec4<R> *>(a.hrec[1])[k];
            ax += (double)hh.x;
            ay += (double)hh.y;
            az += (double)hh.z;
            v[3] += m * ((double)r1.x * (double)hh.x + (double)r1.y * (double)hh.y +
                         (double)r1.z * (double)hh.z + (double)hh.w);
        }
        if (a.acc_pm) {
            ax += a.acc_pm[3 * k];
            ay += a.acc_pm[3 * k + 1];
            az += a.acc_pm[3 * k + 2];
        }
        v[0] += m * ax;
        v[1] += m * ay;
        v[2] += m * az;
    }
    block_sum4(v, partial + 4 * blockIdx.x);
}

__global__ void state_sums_k(State s, int64_t n, double *partial)
{
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const double m = s.m[k];
        const double vx = s.vx[k], vy = s.vy[k], vz = s.vz[k];
        v[0] += m * vx;
        v[1] += m * vy;
        v[2] += m * vz;
        v[3] += 0.5 * m * (vx * vx + vy * vy + vz * vz) + (s.species[k] == CRK_GAS ? m * s.u[k] : 0.0);
    }
    block_sum4(v, partial + 4 * blockIdx.x);
}

__global__ void finish_sums_k(const double *partial, int nblk, double *out)
{
    if (threadIdx.x >= 4) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += partial[4 * b + threadIdx.x];
    out[threadIdx.x] = s;
}

template <typename R>
__global__ void unpermute_outputs_k(PassArgs a, double *acc, double *dudt, double *rho, double *A,
                                    double *B, double *gA, double *gB, int32_t *nc, uint64_t *nh,
                                    int32_t *gc, uint64_t *gh)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.n) return;
    const uint32_t o = a.s.id[k];
    const bool gas = a.s.species[k] == CRK_GAS;
    using R4 = Vec4<R>;
    const R4 g = reinterpret_cast<const R4 *>(a.acc_g)[k];
    R4 hh = {0, 0, 0, 0}, r2 = {0, 0, 0, 0}, r3 = {0, 0, 0, 0}, r4 = {0, 0, 0, 0},
       r5 = {0, 0, 0, 0}, r6 = {0, 0, 0, 0};
    if (gas) {
        hh = reinterpret_cast<const R4 *>(a.acc_h)[k];
        r2 = reinterpret_cast<const R4 *>(a.hrec[2])[k];
        r3 = reinterpret_cast<const R4 *>(a.hrec[3])[k];
        r4 = reinterpret_cast<const R4 *>(a.hrec[4])[k];
        r5 = reinterpret_cast<const R4 *>(a.hrec[5])[k];
        r6 = reinterpret_cast<const R4 *>(a.hrec[6])[k];
    }
    if (acc) {
        double ax = (double)hh.x + (double)g.x, ay = (double)hh.y + (double)g.y,
               az = (double)hh.z + (double)g.z;
        if (a.acc_pm) {
            ax += a.acc_pm[3 * k];
            ay += a.acc_pm[3 * k + 1];
            az += a.acc_pm[3 * k + 2];
        }
        acc[3 * (int64_t)o + 0] = ax;
        acc[3 * (int64_t)o + 1] = ay;
        acc[3 * (int64_t)o + 2] = az;
    }
    if (dudt) dudt[o] = (double)hh.w;
    if (rho) rho[o] = (double)r2.x;
    if (A) A[o] = (double)r2.w;
    if (B) {
        B[3 * (int64_t)o + 0] = (double)r3.x;
        B[3 * (int64_t)o + 1] = (double)r3.y;
        B[3 * (int64_t)o + 2] = (double)r3.z;
    }
    if (gA) {
        gA[3 * (int64_t)o + 0] = (double)r3.w;
        gA[3 * (int64_t)o + 1] = (double)r4.x;
        gA[3 * (int64_t)o + 2] = (double)r4.y;
    }
    if (gB) {
        double* d = gB + 9 * (int64_t)o;
        d[0] = (double)r4.z; d[1] = (double)r4.w;
        d[2] = (double)r5.x; d[3] = (double)r5.y; d[4] = (double)r5.z; d[5] = (double)r5.w;
        d[6] = (double)r6.x; d[7] = (double)r6.y; d[8] = (double)r6.z;
    }
    if (nc) nc[o] = gas && a.nbr_count ? a.nbr_count[k] : 0;
    if (nh) nh[o] = gas && a.nbr_hash ? a.nbr_hash[k] : 0ull;
    if (gc) gc[o] = a.grav_count ? a.grav_count[k] : 0;
    if (gh) gh[o] = a.grav_hash ? a.grav_hash[k] : 0ull;
}

__global__ void unpermute_state_k(State s, int64_t n, double *pos, double *vel, double *u)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t o = s.id[k];
    if (pos) {
        pos[3 * o] = s.x[k];
        pos[3 * o + 1] = s.y[k];
        pos[3 * o + 2] = s.z[k];
    }
    if (vel) {
        vel[3 * o] = s.vx[k];
        vel[3 * o + 1] = s.vy[k];
        vel[3 * o + 2] = s.vz[k];
    }
    if (u) u[o] = s.species[k] == CRK_GAS ? s.u[k] : 0.0;
}

__global__ void load_state_k(State s, int64_t n, const double *pos, const double *vel,
                             const double *mass, const double *u, const double *h,
                             const uint8_t *species, const uint32_t *slot_of)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    s.x[k] = pos[3 * k];
    s.y[k] = pos[3 * k + 1];
    s.z[k] = pos[3 * k + 2];
    s.vx[k] = vel[3 * k];
    s.vy[k] = vel[3 * k + 1];
    s.vz[k] = vel[3 * k + 2];
    const bool gas = species[k] == CRK_GAS;
    s.u[k] = gas ? u[k] : 0.0;
    s.m[k] = mass[k];
    s.h[k] = gas ? h[k] : 0.0;
    s.ax[k] = 0.0;
    s.ay[k] = 0.0;
    s.az[k] = 0.0;
    s.du[k] = 0.0;
    s.species[k] = gas ? (uint8_t)CRK_GAS : (uint8_t)CRK_DM;
    s.slot[k] = slot_of[k];
    s.id[k] = (uint32_t)k;
    s.bin[k] = 0;
}

// Input checks: positions in [0, L) of the particle's box, finite velocity,
// u, positive finite mass, and for gas 0 < 2h < L/2.  Records the smallest
// failing original index.
__global__ void validate_k(State s, const BoxDev *__restrict__ boxes, int64_t n, int *err)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const BoxDev &bx = boxes[s.slot[k]];
    const double L = bx.L;
    bool ok = s.x[k] >= 0.0 && s.x[k] < L && s.y[k] >= 0.0 && s.y[k] < L && s.z[k] >= 0.0 &&
              s.z[k] < L;
    ok = ok && isfinite(s.vx[k]) && isfinite(s.vy[k]) && isfinite(s.vz[k]);
    ok = ok && isfinite(s.m[k]) && s.m[k] > 0.0;
    if (s.species[k] == CRK_GAS) {
        const double H = 2.0 * s.h[k];
        ok = ok && isfinite(s.u[k]) && H > 0.0 && H < 0.5 * L;
    }
    if (!ok) {
        atomicCAS(err, 0, CRK_EINVAL);
        atomicMin(err + 1, (int)s.id[k]);
    }
}

// Replaces x, v, u of the sorted state from arrays in load order.
__global__ void set_state_k(State s, int64_t n, const double *pos, const double *vel,
                            const double *u)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t o = s.id[k];
    if (pos) {
        s.x[k] = pos[3 * o];
        s.y[k] = pos[3 * o + 1];
        s.z[k] = pos[3 * o + 2];
    }
    if (vel) {
        s.vx[k] = vel[3 * o];
        s.vy[k] = vel[3 * o + 1];
        s.vz[k] = vel[3 * o + 2];
    }
    if (u && s.species[k] == CRK_GAS) s.u[k] = u[o];
}

// Copies the state of one box slot out in its own load order (id = index
// within the box).
__global__ void extract_slot_k(State s, int64_t n, uint32_t slot, int64_t n_job, double *pos,
                               double *vel, double *u, double *acc, double *du)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n || s.slot[k] != slot) return;
    const int64_t o = s.id[k];
    if (o >= n_job) return;  // not one of the job's particles
    if (acc) {
        acc[3 * o] = s.ax[k];
        acc[3 * o + 1] = s.ay[k];
        acc[3 * o + 2] = s.az[k];
    }
    if (du) du[o] = s.du[k];
    pos[3 * o] = s.x[k];
    pos[3 * o + 1] = s.y[k];
    pos[3 * o + 2] = s.z[k];
    vel[3 * o] = s.vx[k];
    vel[3 * o + 1] = s.vy[k];
    vel[3 * o + 2] = s.vz[k];
    u[o] = s.species[k] == CRK_GAS ? s.u[k] : 0.0;
}

// The accelerations and du/dt of a force evaluation, set from the caller
// (a job resumed from a snapshot continues with the forces it had).
__global__ void set_forces_k(State s, int64_t n, const double *acc, const double *du)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    s.ax[k] = acc[3 * k];
    s.ay[k] = acc[3 * k + 1];
    s.az[k] = acc[3 * k + 2];
    s.du[k] = s.species[k] == CRK_GAS ? du[k] : 0.0;
}

// Moves the particles of a removed slot to the retired slot, whose box stays
// inactive: the next sort places them last and drops them, and the freed
// slot can take a new job at once.
__global__ void retire_slot_k(uint32_t *slot_of, int64_t n, uint32_t from, uint32_t to)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n && slot_of[k] == from) slot_of[k] = to;
}

__global__ void ds_check_k(uint32_t *dz, int stage, uint32_t cap, const uint32_t *flag)
{
    uint32_t ovf = dz[DZ_OVF];
    if (stage == 0 && dz[DZ_NLEAF_RAW] > cap) ovf |= 1u;
    if (stage == 1 && dz[DZ_NPH] > cap) ovf |= 2u;
    if (stage == 5 && dz[DZ_NPG] > cap) ovf |= 2u;
    if (stage == 3 && dz[DZ_ROWS] > cap) ovf |= 4u;
    if (stage == 4 && flag && *flag) ovf |= 8u;
    if (stage == 6 && flag && *flag) ovf |= 2u;
    dz[DZ_OVF] = ovf;
    if (stage == 0) dz[DZ_NLEAF] = ovf ? 0u : dz[DZ_NLEAF_RAW];
    if (ovf) {
        dz[DZ_NLEAF] = 0u;
        dz[DZ_GGAS] = 0u;
        dz[DZ_GALL] = 0u;
    }
}

}  // namespace

void launch_ds_check(uint32_t *dz, int stage, uint32_t cap, const uint32_t *flag, cudaStream_t st)
{
    ds_check_k<<<1, 1, 0, st>>>(dz, stage, cap, flag);
    note_launches(1);
}

void launch_set_forces(const State &s, int64_t n, const double *acc, const double *du, cudaStream_t st)
{
    if (n <= 0) return;
    set_forces_k<<<nblocks(n), kT, 0, st>>>(s, n, acc, du);
    note_launches(1);
}

void launch_retire_slot(const State &s, int64_t n, uint32_t from, uint32_t to, cudaStream_t st)
{
    if (n <= 0) return;
    retire_slot_k<<<nblocks(n), kT, 0, st>>>(s.slot, n, from, to);
    note_launches(1);
}

void launch_set_state(const State &s, int64_t n, const double *pos, const double *vel,
                      const double *u, cudaStream_t st)
{
    if (n <= 0) return;
    set_state_k<<<nblocks(n), kT, 0, st>>>(s, n, pos, vel, u);
    note_launches(1);
}

void launch_extract_slot(const State &s, int64_t n, uint32_t slot, int64_t n_job, double *pos,
                         double *vel, double *u, double *acc, double *du, cudaStream_t st)
{
    if (n <= 0) return;
    extract_slot_k<<<nblocks(n), kT, 0, st>>>(s, n, slot, n_job, pos, vel, u, acc, du);
    note_launches(1);
}

void launch_validate(const State &s, const BoxDev *boxes, int64_t n, int *err, cudaStream_t st)
{
    if (n <= 0) return;
    validate_k<<<nblocks(n), kT, 0, st>>>(s, boxes, n, err);
    note_launches(1);
}

int sums_blocks(int64_t n)
{
    int64_t b = (n + kT - 1) / kT;
    if (b > 304) b = 304;  // 2 blocks per SM of the 152-SM part
    return b < 1 ? 1 : (int)b;
}

void launch_kick_drift(const State &s, const BoxDev *boxes, int64_t n,
                       unsigned long long *nfloor, cudaStream_t st)
{
    if (n <= 0) return;
    kick_drift_k<<<nblocks(n), kT, 0, st>>>(s, boxes, n, nfloor);
    note_launches(1);
}

void launch_final_kick(const PassArgs &a, int mixed, unsigned long long *nfloor, cudaStream_t st)
{
    if (a.n <= 0) return;
    if (mixed) final_kick_k<float><<<nblocks(a.n), kT, 0, st>>>(a, nfloor);
    else final_kick_k<double><<<nblocks(a.n), kT, 0, st>>>(a, nfloor);
    note_launches(1);
}

void launch_rate_sums(const PassArgs &a, int mixed, double *partial, int nblk, double *out6,
                      cudaStream_t st)
{
    if (a.n <= 0) {
        cudaMemsetAsync(out6, 0, 4 * sizeof(double), st);
        return;
    }
    if (mixed) rate_sums_k<float><<<nblk, kT, 0, st>>>(a, partial);
    else rate_sums_k<double><<<nblk, kT, 0, st>>>(a, partial);
    note_launches(1);
    finish_sums_k<<<1, 32, 0, st>>>(partial, nblk, out6);
    note_launches(1);
}

void launch_state_sums(const State &s, int64_t n, double *partial, int nblk, double *out6,
                       cudaStream_t st)
{
    if (n <= 0) {
        cudaMemsetAsync(out6, 0, 4 * sizeof(double), st);
        return;
    }
    state_sums_k<<<nblk, kT, 0, st>>>(s, n, partial);
    note_launches(1);
    finish_sums_k<<<1, 32, 0, st>>>(partial, nblk, out6);
    note_launches(1);
}

void launch_unpermute_outputs(const PassArgs &a, int mixed, double *acc, double *dudt,
                              double *rho, double *A, double *B, double *gA, double *gB,
                              int32_t *nc, uint64_t *nh, int32_t *gc, uint64_t *gh,
                              cudaStream_t st)
{
    if (a.n <= 0) return;
    if (mixed)
        unpermute_outputs_k<float><<<nblocks(a.n), kT, 0, st>>>(a, acc, dudt, rho, A, B, gA, gB,
                                                                nc, nh, gc, gh);
    else
        unpermute_outputs_k<double><<<nblocks(a.n), kT, 0, st>>>(a, acc, dudt, rho, A, B, gA, gB,
                                                                 nc, nh, gc, gh);
}

void launch_unpermute_state(const State &s, int64_t n, double *pos, double *vel, double *u,
                            cudaStream_t st)
{
    if (n <= 0) return;
    unpermute_state_k<<<nblocks(n), kT, 0, st>>>(s, n, pos, vel, u);
    note_launches(1);
}

void launch_load_state(const State &s, int64_t n, const double *pos, const double *vel,
                       const double *mass, const double *u, const double *h,
                       const uint8_t *species, const uint32_t *slot_of, cudaStream_t st)
{
    if (n <= 0) return;
    load_state_k<<<nblocks(n), kT, 0, st>>>(s, n, pos, vel, mass, u, h, species, slot_of);
    note_launches(1);
}

}  // namespace crk
