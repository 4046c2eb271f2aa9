// Hierarchical (block) time steps: particles in power-of-two timestep bins,
// forces evaluated only where a particle's step ends (paper Sec. II and
// IV-B1: adaptive integration with particles grouped into timestep bins; only
// the active leaves are updated in a substep, the leaves themselves are kept
// and their boxes grow over the long step).
//
// A long step D_t is cut into 2^depth substeps of length d; a particle in bin
// b takes steps of L_b = 2^(depth - b) substeps that start at multiples of
// L_b.  Substep s: opening kick of the particles whose step starts at s, drift
// of all, forces at t_(s+1) for the particles whose step ends at s + 1 (the
// active ones: bin >= depth - trailing_zeros(s + 1)), closing kick of those
// and a new bin for each from the acceleration and Courant criteria.  Every
// product and sum of the state update is rounded on its own (FP64).
#include "crk_internal.h"

namespace crk {

namespace {

constexpr int kT = 256;

inline unsigned nblocks(int64_t n) { return (unsigned)((n + kT - 1) / kT); }

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

__device__ __forceinline__ double floor_u(double u, double fl, unsigned long long *nfloor)
{
    if (u < fl) {
        atomicAdd(nfloor, 1ull);
        return fl;
    }
    return u;
}

// Opening kick of the particles whose step starts at substep s, then the
// drift of every particle by d.
__global__ void kick_drift_bins_k(State s, const BoxDev *__restrict__ boxes, int64_t n, int sub, int depth,
                                  double d, unsigned long long *nfloor)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const BoxDev &bx = boxes[s.slot[k]];
    const int Lb = 1 << (depth - (int)s.bin[k]);
    double vx = s.vx[k], vy = s.vy[k], vz = s.vz[k];
    if (sub % Lb == 0) {
        const double hdt = __dmul_rn((double)Lb, 0.5 * d);  // dt_b / 2, exact
        vx = __dadd_rn(vx, __dmul_rn(hdt, s.ax[k]));
        vy = __dadd_rn(vy, __dmul_rn(hdt, s.ay[k]));
        vz = __dadd_rn(vz, __dmul_rn(hdt, s.az[k]));
        s.vx[k] = vx;
        s.vy[k] = vy;
        s.vz[k] = vz;
        if (s.species[k] == CRK_GAS) s.u[k] = floor_u(__dadd_rn(s.u[k], __dmul_rn(hdt, s.du[k])), bx.u_floor, nfloor);
    }
    s.x[k] = drift_wrap(s.x[k], d, vx, bx.L);
    s.y[k] = drift_wrap(s.y[k], d, vy, bx.L);
    s.z[k] = drift_wrap(s.z[k], d, vz, bx.L);
}

// Bin of a particle from its acceleration and (gas) u: the shallowest b with
// D_t / 2^b <= min(sqrt(2 eta eps / |a|), courant h / c), at most depth, and
// no shallower than b_sync (a particle only joins a bin whose steps start now).
__device__ __forceinline__ int bin_of(double ax, double ay, double az, double u, double h, bool gas,
                                      const BoxDev &bx, double dt_long, int depth, double eta,
                                      double courant, int b_sync)
{
    const double amag = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(ax, ax), __dmul_rn(ay, ay)), __dmul_rn(az, az)));
    double dt = __longlong_as_double(0x7ff0000000000000ll);  // +inf
    if (bx.eps_soft > 0.0 && amag > 0.0) dt = sqrt(__ddiv_rn(__dmul_rn(2.0 * eta, bx.eps_soft), amag));
    if (gas && u > 0.0) {
        const double c = sqrt(__dmul_rn(__dmul_rn(bx.gamma, bx.gamma - 1.0), u));
        dt = fmin(dt, __ddiv_rn(__dmul_rn(courant, h), c));
    }
    int b = 0;
    for (int k = 0; k < depth; ++k)
        if (ldexp(dt_long, -k) > dt) b = k + 1;
    return b > b_sync ? b : b_sync;
}

// Closing kick of the particles active at the end of substep s with the
// accelerations just computed, then their new bins.  Inactive particles keep
// the state and the rates of their last evaluation.
template <typename R>
__global__ void close_bins_k(PassArgs a, int sub, int depth, double d, double dt_long, double eta,
                             double courant, int b_sync, unsigned long long *nfloor,
                             unsigned long long *nactive)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.n) return;
    const int Lb = 1 << (depth - (int)a.s.bin[k]);
    const bool act = (sub + 1) % Lb == 0;
    const unsigned bal = __ballot_sync(__activemask(), act);
    if (nactive && (threadIdx.x & 31u) == (unsigned)(__ffs(__activemask()) - 1))
        atomicAdd(nactive, (unsigned long long)__popc(bal));
    if (!act) return;
    const BoxDev &bx = a.boxes[a.s.slot[k]];
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
    const double hdt = __dmul_rn((double)Lb, 0.5 * d);
    a.s.vx[k] = __dadd_rn(a.s.vx[k], __dmul_rn(hdt, ax));
    a.s.vy[k] = __dadd_rn(a.s.vy[k], __dmul_rn(hdt, ay));
    a.s.vz[k] = __dadd_rn(a.s.vz[k], __dmul_rn(hdt, az));
    double u = 0.0;
    if (gas) {
        u = floor_u(__dadd_rn(a.s.u[k], __dmul_rn(hdt, du)), bx.u_floor, nfloor);
        a.s.u[k] = u;
    }
    a.s.ax[k] = ax;
    a.s.ay[k] = ay;
    a.s.az[k] = az;
    a.s.du[k] = du;
    a.s.bin[k] = (uint8_t)bin_of(ax, ay, az, u, a.s.h[k], gas, bx, dt_long, depth, eta, courant, b_sync);
}

// Bins of every particle from the stored rates (the start of a long step).
__global__ void assign_bins_k(State s, const BoxDev *__restrict__ boxes, int64_t n, double dt_long, int depth,
                              double eta, double courant)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const bool gas = s.species[k] == CRK_GAS;
    s.bin[k] = (uint8_t)bin_of(s.ax[k], s.ay[k], s.az[k], gas ? s.u[k] : 0.0, s.h[k], gas, boxes[s.slot[k]],
                               dt_long, depth, eta, courant, 0);
}

// Leaves holding a particle active at the end of the substep (bin >= bmin).
__global__ void leaf_active_k(Leaves lv, int nleaf, const uint8_t *__restrict__ bin, int bmin, uint8_t *flag)
{
    const int L = blockIdx.x * blockDim.x + threadIdx.x;
    if (L >= nleaf) return;
    const uint32_t s0 = lv.start[L], c = lv.count[L];
    uint8_t f = 0;
    for (uint32_t k = 0; k < c && !f; ++k) f = bin[s0 + k] >= bmin;
    flag[L] = f;
}

// out[I] = in[I] or in[J] for a J of I's hydro leaf-pair row (the rows are
// symmetric): the leaves whose particles a flagged leaf's targets read.
__global__ void leaf_expand_k(const uint32_t *__restrict__ row, const uint32_t *__restrict__ col, int nleaf,
                              const uint8_t *__restrict__ in, uint8_t *out)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nleaf) return;
    uint8_t f = in[I];
    for (uint32_t p = row[I]; p < row[I + 1] && !f; ++p) f = in[col[p]];
    out[I] = f;
}

// Keep-flags of the work items of a group list (item = (leaf, offset)):
// leaf flagged, and not flagged in exclude (optional).
__global__ void group_flags_k(const uint2 *__restrict__ groups, uint32_t n, const uint8_t *__restrict__ leaf_flag,
                              const uint8_t *__restrict__ exclude, uint32_t *keep)
{
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const uint32_t L = groups[g].x;
    keep[g] = leaf_flag[L] && !(exclude && exclude[L]);
}

// Stable compaction of the kept items; map (optional) gets each kept item's
// index in the source list.
__global__ void group_compact_k(const uint2 *__restrict__ groups, uint32_t n, const uint32_t *__restrict__ keep,
                                const uint32_t *__restrict__ pos, uint2 *out, uint32_t *map)
{
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n || !keep[g]) return;
    out[pos[g]] = groups[g];
    if (map) map[pos[g]] = g;
}

// Long-range kick of every particle: v += hdt a_mesh (FP64, each product and
// sum rounded on its own).
__global__ void pm_kick_k(State s, const double *__restrict__ acc, int64_t n, double hdt)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    s.vx[k] = __dadd_rn(s.vx[k], __dmul_rn(hdt, acc[3 * k]));
    s.vy[k] = __dadd_rn(s.vy[k], __dmul_rn(hdt, acc[3 * k + 1]));
    s.vz[k] = __dadd_rn(s.vz[k], __dmul_rn(hdt, acc[3 * k + 2]));
}

__global__ void unpermute_bins_k(State s, int64_t n, uint8_t *out)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    out[s.id[k]] = s.bin[k];
}

}  // namespace

void launch_kick_drift_bins(const State &s, const BoxDev *boxes, int64_t n, int sub, int depth, double d,
                            unsigned long long *nfloor, cudaStream_t st)
{
    if (n <= 0) return;
    kick_drift_bins_k<<<nblocks(n), kT, 0, st>>>(s, boxes, n, sub, depth, d, nfloor);
    note_launches(1);
}

void launch_close_bins(const PassArgs &a, int mixed, int sub, int depth, double d, double dt_long, double eta,
                       double courant, int b_sync, unsigned long long *nfloor, unsigned long long *nactive,
                       cudaStream_t st)
{
    if (a.n <= 0) return;
    if (mixed)
        close_bins_k<float><<<nblocks(a.n), kT, 0, st>>>(a, sub, depth, d, dt_long, eta, courant, b_sync, nfloor,
                                                        nactive);
    else
        close_bins_k<double><<<nblocks(a.n), kT, 0, st>>>(a, sub, depth, d, dt_long, eta, courant, b_sync, nfloor,
                                                         nactive);
    note_launches(1);
}

void launch_assign_bins(const State &s, const BoxDev *boxes, int64_t n, double dt_long, int depth, double eta,
                        double courant, cudaStream_t st)
{
    if (n <= 0) return;
    assign_bins_k<<<nblocks(n), kT, 0, st>>>(s, boxes, n, dt_long, depth, eta, courant);
    note_launches(1);
}

void launch_leaf_active(const Leaves &lv, int nleaf, const uint8_t *bin, int bmin, uint8_t *flag, cudaStream_t st)
{
    if (nleaf <= 0) return;
    leaf_active_k<<<nblocks(nleaf), kT, 0, st>>>(lv, nleaf, bin, bmin, flag);
    note_launches(1);
}

void launch_leaf_expand(const uint32_t *row, const uint32_t *col, int nleaf, const uint8_t *in, uint8_t *out,
                        cudaStream_t st)
{
    if (nleaf <= 0) return;
    leaf_expand_k<<<nblocks(nleaf), kT, 0, st>>>(row, col, nleaf, in, out);
    note_launches(1);
}

void launch_group_select(const uint2 *groups, uint32_t n, const uint8_t *leaf_flag, uint32_t *keep, uint32_t *pos,
                         uint32_t *total, uint32_t *tmp, uint2 *out, uint32_t *map, cudaStream_t st,
                         const uint8_t *exclude)
{
    if (n == 0) {
        cudaMemsetAsync(total, 0, sizeof(uint32_t), st);
        return;
    }
    group_flags_k<<<nblocks(n), kT, 0, st>>>(groups, n, leaf_flag, exclude, keep);
    scan_exclusive_u32(keep, pos, n, total, tmp, st);
    group_compact_k<<<nblocks(n), kT, 0, st>>>(groups, n, keep, pos, out, map);
    note_launches(2);
}

void launch_pm_kick(const State &s, const double *acc, int64_t n, double hdt, cudaStream_t st)
{
    if (n <= 0) return;
    pm_kick_k<<<nblocks(n), kT, 0, st>>>(s, acc, n, hdt);
    note_launches(1);
}

void launch_unpermute_bins(const State &s, int64_t n, uint8_t *out, cudaStream_t st)
{
    if (n <= 0) return;
    unpermute_bins_k<<<nblocks(n), kT, 0, st>>>(s, n, out);
    note_launches(1);
}

}  // namespace crk
