// Spatial structure of the short-range solver (paper Sec. IV-B1, "GPU Tree
// Solver"): particles are binned by a Morton key, cut into base leaves of at
// most leaf_cap particles that never straddle a chaining-mesh bin, and the
// leaf-pair interaction lists are produced from conservative bounding-box
// gaps.  Only the base leaves are kept, as in the paper; a throw-away implicit
// binary hierarchy over the Morton-ordered leaves serves the pair search.
//
// Every kernel here is memory-bound: coalesced SoA loads, one pass per
// array, grid sizes in multiples of the SM count where the work is flat.
#include "crk_internal.h"

#include <cfloat>

namespace crk {

namespace {

constexpr int kT = 256;            // threads per block for flat kernels
constexpr int kItems = 16;         // items per thread in scan / sort tiles
constexpr int kTile = kT * kItems; // 4096
static_assert(kTile == kSortTile, "scratch sizing of the scan and sort tiles");

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v)
{
    const uint32_t lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= (uint32_t)o) v += t;
    }
    return v;
}

// Exclusive block scan of one value per thread (blockDim.x == kT or 1024).
template <int NT>
__device__ uint32_t block_excl_scan(uint32_t v, uint32_t *total)
{
    __shared__ uint32_t wsum[NT / 32];
    const uint32_t lane = lane_id(), w = threadIdx.x >> 5;
    uint32_t inc = warp_incl_scan(v);
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint32_t s = (lane < NT / 32) ? wsum[lane] : 0u;
        uint32_t si = warp_incl_scan(s);
        if (lane < NT / 32) wsum[lane] = si - s;
        if (lane == NT / 32 - 1 && total) *total = si;
    }
    __syncthreads();
    uint32_t r = inc - v + wsum[w];
    __syncthreads();
    return r;
}

__global__ void scan_reduce_k(const uint32_t *__restrict__ in, int64_t n, uint32_t *part)
{
    const int64_t base = (int64_t)blockIdx.x * kTile;
    uint32_t s = 0;
    for (int i = threadIdx.x; i < kTile; i += kT) {
        int64_t k = base + i;
        if (k < n) s += in[k];
    }
    __shared__ uint32_t tot;
    block_excl_scan<kT>(s, &tot);
    __syncthreads();
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void scan_partials_k(uint32_t *part, int64_t nb, uint32_t *total)
{
    __shared__ uint32_t chunk_total;
    uint32_t running = 0;
    for (int64_t c = 0; c < nb; c += 1024) {
        int64_t k = c + threadIdx.x;
        uint32_t v = (k < nb) ? part[k] : 0u;
        uint32_t ex = block_excl_scan<1024>(v, &chunk_total);
        __syncthreads();
        if (k < nb) part[k] = running + ex;
        running += chunk_total;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = running;
}

__global__ void scan_down_k(const uint32_t *in, uint32_t *out, int64_t n, const uint32_t *part)
{
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
    uint32_t v[kItems];
    uint32_t s = 0;
#pragma unroll
    for (int t = 0; t < kItems; ++t) {
        int64_t k = base + t;
        v[t] = (k < n) ? in[k] : 0u;
        s += v[t];
    }
    uint32_t ex = block_excl_scan<kT>(s, nullptr) + part[blockIdx.x];
#pragma unroll
    for (int t = 0; t < kItems; ++t) {
        int64_t k = base + t;
        if (k < n) out[k] = ex;
        ex += v[t];
    }
}

// ---------------------------------------------------------------- radix sort
__global__ void radix_hist_k(const uint64_t *__restrict__ keys, int64_t n, int shift,
                             uint32_t *counts, int64_t nb)
{
    __shared__ uint32_t hist[256];
    hist[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile;
    for (int i = threadIdx.x; i < kTile; i += kT) {
        int64_t k = base + i;
        bool valid = k < n;
        uint32_t d = valid ? (uint32_t)((keys[k] >> shift) & 255u) : 256u;
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        if (valid && lane_id() == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&hist[d], __popc(peers));
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * nb + blockIdx.x] = hist[threadIdx.x];
}

// Stable scatter: items of a tile are ranked in order (round by round, warp
// by warp, lane by lane) so equal digits keep their input order.
__global__ void radix_scatter_k(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                                uint64_t *kout, uint32_t *vout, int64_t n, int shift,
                                const uint32_t *__restrict__ offs, int64_t nb)
{
    __shared__ uint32_t run[256];
    __shared__ uint32_t wcnt[kT / 32][256];
    const uint32_t tid = threadIdx.x, w = tid >> 5, lane = lane_id();
    run[tid] = offs[(int64_t)tid * nb + blockIdx.x];
    const uint32_t lt = (1u << lane) - 1u;
    const int64_t base = (int64_t)blockIdx.x * kTile;
    for (int r = 0; r < kItems; ++r) {
#pragma unroll
        for (int q = 0; q < kT / 32; ++q) wcnt[q][tid] = 0;
        __syncthreads();
        int64_t k = base + (int64_t)r * kT + tid;
        bool valid = k < n;
        uint64_t key = valid ? kin[k] : 0ull;
        uint32_t val = valid ? vin[k] : 0u;
        uint32_t d = valid ? (uint32_t)((key >> shift) & 255u) : 256u;
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t rank = __popc(peers & lt);
        if (valid && lane == (uint32_t)(__ffs(peers) - 1)) wcnt[w][d] = __popc(peers);
        __syncthreads();
        {
            uint32_t running = run[tid];
#pragma unroll
            for (int q = 0; q < kT / 32; ++q) {
                uint32_t c = wcnt[q][tid];
                wcnt[q][tid] = running;
                running += c;
            }
            run[tid] = running;
        }
        __syncthreads();
        if (valid) {
            uint32_t pos = wcnt[w][d] + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- keys
__device__ __forceinline__ uint64_t spread3(uint64_t v)
{
    v &= 0x1fffffull;
    v = (v | v << 32) & 0x1f00000000ffffull;
    v = (v | v << 16) & 0x1f0000ff0000ffull;
    v = (v | v << 8) & 0x100f00f00f00f00full;
    v = (v | v << 4) & 0x10c30c30c30c30c3ull;
    v = (v | v << 2) & 0x1249249249249249ull;
    return v;
}

__device__ __forceinline__ uint32_t cell21(double x, double L)
{
    double c = x / L * 2097152.0;
    if (!(c >= 0.0)) c = 0.0;
    uint32_t ci = (uint32_t)c;
    return ci > 2097151u ? 2097151u : ci;
}

__global__ void morton_keys_k(State s, const BoxDev *__restrict__ boxes, int64_t n, int sb,
                              uint64_t *keys, uint32_t *idx)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    uint32_t slot = s.slot[k];
    if (!boxes[slot].active) {
        keys[k] = ~0ull;
        idx[k] = (uint32_t)k;
        return;
    }
    double L = boxes[slot].L;
    uint64_t m = spread3(cell21(s.x[k], L)) | (spread3(cell21(s.y[k], L)) << 1) |
                 (spread3(cell21(s.z[k], L)) << 2);
    uint64_t sp = (uint64_t)(s.species[k] & 1u);
    uint64_t key;
    if (sb == 0) key = (sp << 63) | m;
    else key = ((uint64_t)slot << (64 - sb)) | (sp << (63 - sb)) | (m >> sb);
    keys[k] = key;
    idx[k] = (uint32_t)k;
}

__global__ void permute_k(State a, State b, const uint32_t *__restrict__ perm, int64_t n)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    uint32_t p = perm[k];
    b.x[k] = a.x[p]; b.y[k] = a.y[p]; b.z[k] = a.z[p];
    b.vx[k] = a.vx[p]; b.vy[k] = a.vy[p]; b.vz[k] = a.vz[p];
    b.u[k] = a.u[p]; b.m[k] = a.m[p]; b.h[k] = a.h[p];
    b.ax[k] = a.ax[p]; b.ay[k] = a.ay[p]; b.az[k] = a.az[p]; b.du[k] = a.du[p];
    b.species[k] = a.species[p]; b.slot[k] = a.slot[p]; b.id[k] = a.id[p]; b.bin[k] = a.bin[p];
}

// ---------------------------------------------------------------- leaves
// True when the Morton cell of particle k at key shift s (the prefix
// key >> s) holds at most cap particles; then lo is its first particle.
// Both ends of such a cell lie within cap positions of k, so every probe
// stays in [k - cap, k + cap].
__device__ __forceinline__ bool cell_fits(const uint64_t *__restrict__ keys, int64_t n, int64_t k,
                                          uint64_t key, int s, int cap, int64_t &lo)
{
    const uint64_t p = key >> s;
    if (k >= cap && (keys[k - cap] >> s) == p) return false;
    int64_t a = k - cap + 1 > 0 ? k - cap + 1 : 0, b = k;
    while (a < b) {
        const int64_t mid = (a + b) >> 1;
        if ((keys[mid] >> s) < p) a = mid + 1;
        else b = mid;
    }
    lo = a;
    return !(lo + cap < n && (keys[lo + cap] >> s) == p);
}

// First index in [a, b) whose key prefix (key >> s) is >= p (keys sorted).
__device__ __forceinline__ int64_t prefix_lower_bound(const uint64_t *__restrict__ keys, int64_t a, int64_t b,
                                                      int s, uint64_t p)
{
    while (a < b) {
        const int64_t mid = (a + b) >> 1;
        if ((keys[mid] >> s) < p) a = mid + 1;
        else b = mid;
    }
    return a;
}

// Leaf cells are packed with their siblings: the children of one octree
// cell that is too large to be a leaf are taken in Morton order, and runs of
// consecutive children that each fit (at most cap particles) are packed
// greedily into leaves of at most cap particles; a child that does not fit
// (it is cut into deeper leaves) ends a run.  True when the leaf cell of
// particle k (its first particle, at shift s, parent at shift s + 3, cell
// range [lo, hi)) starts a new leaf.  Every probe stays inside the parent's
// range, which lies in [0, hi].
__device__ bool starts_packed_leaf(const uint64_t *__restrict__ keys, int64_t lo, int64_t hi, uint64_t key, int s,
                                   int cap)
{
    const uint64_t parent = key >> (s + 3);
    const uint32_t own = (uint32_t)((key >> s) & 7u);
    int64_t c0 = prefix_lower_bound(keys, 0, lo, s + 3, parent);   // the parent's first particle
    uint32_t acc = 0;
    bool start = true;
    for (uint32_t c = 0; c <= own; ++c) {
        const int64_t c1 = c == own ? hi : prefix_lower_bound(keys, c0, lo, s, (parent << 3) | (c + 1));
        const uint32_t cnt = (uint32_t)(c1 - c0);
        c0 = c1;
        if (cnt == 0) continue;
        if (cnt > (uint32_t)cap) {
            acc = 0;
            continue;
        }
        start = acc == 0 || acc + cnt > (uint32_t)cap;
        acc = start ? cnt : acc + cnt;
    }
    return start;
}

// Leaves: the coarsest Morton cells, at or below the box's chaining-mesh
// bin, that hold at most cap particles of one (box, species), packed with
// their small siblings (starts_packed_leaf), so that leaves are compact runs
// of Morton order that rarely fall far below cap.  Cells are found per
// particle by a binary search over the levels (a cell's count only shrinks
// with depth).  Particles that share even the finest cell are cut by count.
// flags[k] = 1 where a leaf starts.  The keys are sorted on their bits from
// first_bit up only, so levels whose cells need lower bits are not used: a
// cell at the deepest sorted level that still holds more than cap particles
// is cut by count.  stats[0] gets the deepest level used, stats[1] is set
// when such a cut happened above levels that exist.
__global__ void leaf_flags_k(const uint64_t *__restrict__ keys, int sb,
                             const BoxDev *__restrict__ boxes, int64_t n, int cap, uint32_t *flags,
                             int first_bit, uint32_t *stats)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const uint64_t key = keys[k];
    const uint32_t slot = sb ? (uint32_t)(key >> (64 - sb)) : 0u;
    const int s0 = boxes[slot].cm_shift;     // shift of the chaining-mesh bin
    const int lall = s0 / 3;                 // deepest level with a non-negative shift
    const int lsorted = (s0 - first_bit) / 3;
    const int lmax = lall < lsorted ? lall : lsorted;
    int la = 0, lb = lmax + 1;
    int64_t lo = 0;
    while (la < lb) {
        const int mid = (la + lb) >> 1;
        if (cell_fits(keys, n, k, key, s0 - 3 * mid, cap, lo)) lb = mid;
        else la = mid + 1;
    }
    if (la <= lmax) {
        const int s = s0 - 3 * la;
        cell_fits(keys, n, k, key, s, cap, lo);
        uint32_t f = 0u;
        if (k == lo) {
            atomicMax(stats, (uint32_t)la);
            f = 1u;
            if (la >= 1) {
                // the cell's end: it holds at most cap particles
                const int64_t hi = prefix_lower_bound(keys, k, k + cap < n ? k + cap + 1 : n, s, (key >> s) + 1);
                f = starts_packed_leaf(keys, lo, hi, key, s, cap) ? 1u : 0u;
            }
        }
        flags[k] = f;
    } else {
        if (k % cap == 0 && lmax < lall) atomicOr(stats + 1, 1u);
        const int s = s0 - 3 * lmax;
        const uint64_t g = key >> s;
        int64_t a = 0, b = k;
        while (a < b) {
            const int64_t mid = (a + b) >> 1;
            if ((keys[mid] >> s) < g) a = mid + 1;
            else b = mid;
        }
        flags[k] = ((k - a) % cap) == 0 ? 1u : 0u;
    }
}

// Leaves whose index reaches `cap` (the leaf arrays' capacity) are not
// written; nl_dev (optional) holds the leaf count on the device, capped at
// the capacity by the caller when it overflows.
__device__ __forceinline__ int leaves_of(int nleaf, const uint32_t *nl_dev)
{
    return nl_dev ? (int)min((uint32_t)nleaf, *nl_dev) : nleaf;
}

__global__ void leaf_setup_k(const uint32_t *__restrict__ flags, const uint32_t *__restrict__ scan,
                             int64_t n, uint32_t cap, uint32_t *start)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    if (flags[k] && scan[k] < cap) start[scan[k]] = (uint32_t)k;
}

__global__ void leaf_count_k(Leaves lv, int nleaf, int64_t n, const uint32_t *nl_dev)
{
    int L = blockIdx.x * blockDim.x + threadIdx.x;
    const int nl = leaves_of(nleaf, nl_dev);
    if (L >= nl) return;
    uint32_t end = (L + 1 < nl) ? lv.start[L + 1] : (uint32_t)n;
    lv.count[L] = end - lv.start[L];
}

__device__ __forceinline__ double wmin(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double wmax(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float wminf(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float wmaxf(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// One warp per leaf: FP64 bounds, centre, half extents (rounded up), the
// leaf's largest kernel support, the level-0 node, and the position-mass
// records of its particles (leaf-relative FP32 in the mixed form, absolute
// FP64 in the plain form).
// Offset of a coordinate from a leaf's reference particle, wrapped once: a
// leaf whose particles drifted across a periodic face keeps a compact box
// (its box may then reach past [0, L); every user wraps differences).
__device__ __forceinline__ double leaf_offset(double x, double ref, double L)
{
    double d = x - ref;
    if (d >= 0.5 * L) d -= L;
    else if (d < -0.5 * L) d += L;
    return d;
}

template <int MIXED>
__global__ void leaf_bounds_k(State s, const BoxDev *__restrict__ boxes, Leaves lv, int nleaf, void *pm,
                              Nodes nd, const uint32_t *nl_dev)
{
    const int w = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const uint32_t lane = lane_id();
    if (w >= nleaf) return;
    if (w >= leaves_of(nleaf, nl_dev)) {
        // an unused slot of the leaf arrays (capacity beyond the leaf count):
        // an empty leaf whose node box is inverted and belongs to no box, so
        // that every walk of the hierarchy passes it by
        if (lane == 0) {
            lv.count[w] = 0;
            lv.species[w] = 0xffu;
            lv.hmax[w] = 0.f;
            nd.lo[w] = make_float4(1e30f, 1e30f, 1e30f, 0.f);
            nd.hi[w] = make_float4(-1e30f, -1e30f, -1e30f, __int_as_float(-2));
        }
        return;
    }
    const uint32_t s0 = lv.start[w], c = lv.count[w];
    const double Lb = boxes[s.slot[s0]].L;
    // positions relative to the leaf's first particle (leaves built from a
    // Morton cell never straddle a face; leaves kept between rebuilds may);
    // particle 32 ch + lane of the leaf is this lane's ch-th (c <= 128)
    const double ref[3] = {s.x[s0], s.y[s0], s.z[s0]};
    double d[kChunks][3];
    double lo[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, hi[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
    float hm = 0.f;  // max 2h, rounded up (rounding is monotonic: the max of the rounded values)
#pragma unroll
    for (int ch = 0; ch < kChunks; ++ch) {
        const uint32_t t = 32u * ch + lane;
        if (t < c) {
            const uint32_t i = s0 + t;
            d[ch][0] = leaf_offset(s.x[i], ref[0], Lb);
            d[ch][1] = leaf_offset(s.y[i], ref[1], Lb);
            d[ch][2] = leaf_offset(s.z[i], ref[2], Lb);
#pragma unroll
            for (int a = 0; a < 3; ++a) { lo[a] = fmin(lo[a], d[ch][a]); hi[a] = fmax(hi[a], d[ch][a]); }
            if (s.species[i] == CRK_GAS) hm = fmaxf(hm, __double2float_ru(2.0 * s.h[i]));
        } else {
            d[ch][0] = d[ch][1] = d[ch][2] = 0.0;
        }
    }
    double cen[3], mid[3];
    float ext[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lo[a] = wmin(lo[a]);
        hi[a] = wmax(hi[a]);
        mid[a] = 0.5 * (lo[a] + hi[a]);          // centre relative to the reference
        cen[a] = ref[a] + mid[a];
        ext[a] = __double2float_ru(fmax(hi[a] - mid[a], mid[a] - lo[a]));
    }
    hm = wmaxf(hm);
    if (lane == 0) {
        lv.cx[w] = cen[0]; lv.cy[w] = cen[1]; lv.cz[w] = cen[2];
        lv.ex[w] = ext[0]; lv.ey[w] = ext[1]; lv.ez[w] = ext[2];
        lv.hmax[w] = hm;
        lv.slot[w] = s.slot[s0];
        lv.species[w] = s.species[s0];
        nd.lo[w] = make_float4(__double2float_rd(ref[0] + lo[0]), __double2float_rd(ref[1] + lo[1]),
                               __double2float_rd(ref[2] + lo[2]), hm);
        nd.hi[w] = make_float4(__double2float_ru(ref[0] + hi[0]), __double2float_ru(ref[1] + hi[1]),
                               __double2float_ru(ref[2] + hi[2]), __int_as_float((int32_t)s.slot[s0]));
    }
    // Boxes of the 32-particle chunks (particle t of the leaf is in chunk t/32),
    // relative to the leaf centre, rounded outward; empty chunks get an
    // inverted box that is never in range.  Rounding is monotonic, so the
    // FP32 minimum of the values rounded down is the FP64 minimum rounded
    // down (and likewise up for the maximum): the reductions run in FP32.
#pragma unroll
    for (int ch = 0; ch < kChunks; ++ch) {
        const bool in = 32u * ch + lane < c;
        const double px = d[ch][0] - mid[0], py = d[ch][1] - mid[1], pz = d[ch][2] - mid[2];
        const float lx = wminf(in ? __double2float_rd(px) : FLT_MAX), hx = wmaxf(in ? __double2float_ru(px) : -FLT_MAX);
        const float ly = wminf(in ? __double2float_rd(py) : FLT_MAX), hy = wmaxf(in ? __double2float_ru(py) : -FLT_MAX);
        const float lz = wminf(in ? __double2float_rd(pz) : FLT_MAX), hz = wmaxf(in ? __double2float_ru(pz) : -FLT_MAX);
        if (lane == 0) {
            const bool any = 32u * ch < c;
            lv.clo[(size_t)w * kChunks + ch] =
                any ? make_float4(lx, ly, lz, 0.f) : make_float4(1e30f, 1e30f, 1e30f, 0.f);
            lv.chi[(size_t)w * kChunks + ch] =
                any ? make_float4(hx, hy, hz, 0.f) : make_float4(-1e30f, -1e30f, -1e30f, 0.f);
        }
        if (in) {
            const uint32_t i = s0 + 32u * ch + lane;
            if (MIXED) {
                float4 r;
                r.x = (float)px;
                r.y = (float)py;
                r.z = (float)pz;
                r.w = (float)s.m[i];
                reinterpret_cast<float4 *>(pm)[i] = r;
            } else {
                Vec4<double> r;
                r.x = s.x[i]; r.y = s.y[i]; r.z = s.z[i]; r.w = s.m[i];
                reinterpret_cast<Vec4<double> *>(pm)[i] = r;
            }
        }
    }
}

__global__ void node_level_k(Nodes nd, int64_t oc, int64_t ncld, int64_t op, int64_t npar)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= npar) return;
    int64_t c0 = oc + 2 * k, c1 = oc + 2 * k + 1;
    float4 lo = nd.lo[c0], hi = nd.hi[c0];
    if (2 * k + 1 < ncld) {
        const float4 l1 = nd.lo[c1], h1 = nd.hi[c1];
        lo.x = fminf(lo.x, l1.x); lo.y = fminf(lo.y, l1.y); lo.z = fminf(lo.z, l1.z);
        lo.w = fmaxf(lo.w, l1.w);  // max H
        hi.x = fmaxf(hi.x, h1.x); hi.y = fmaxf(hi.y, h1.y); hi.z = fmaxf(hi.z, h1.z);
        if (__float_as_int(h1.w) != __float_as_int(hi.w)) hi.w = __int_as_float(-1);
    }
    int64_t o = op + k;
    nd.lo[o] = lo;
    nd.hi[o] = hi;
}

// Depth-first walk of the leaf hierarchy from leaf I, left child first, so a
// row lists its neighbour leaves in ascending order whatever else is loaded.
// A node is kept when its periodic box gap to I is below the pair radius R
// (hydro: max of the two largest supports; gravity: r_cut), widened by a
// small relative and absolute margin so FP32 rounding never drops a pair.
// Frame of leaf pair (I, J) for the mixed-form pair passes: the shift
// s = wrap(c_J - c_I) formed in FP64 and rounded to FP32, and the bound
// mag = sum over axes of |s| + e_I + e_J (plus L when a per-pair wrap is still
// needed, flagged by a negative sign) that sizes the FP32 guard band.
__device__ __forceinline__ float4 pair_frame(const Leaves &lv, int I, int J, double L)
{
    const double hL = 0.5 * L;
    double d[3] = {lv.cx[J] - lv.cx[I], lv.cy[J] - lv.cy[I], lv.cz[J] - lv.cz[I]};
    float s[3];
    const float e[3] = {lv.ex[I] + lv.ex[J], lv.ey[I] + lv.ey[J], lv.ez[I] + lv.ez[J]};
    bool wrap = false;
    float mag = 0.f;
    const float lim = (float)hL * (1.0f - 1e-6f);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (d[a] >= hL) d[a] -= L;
        else if (d[a] < -hL) d[a] += L;
        s[a] = (float)d[a];
        const float m = fabsf(s[a]) + e[a];
        wrap = wrap || (m >= lim);
        mag += m;
    }
    if (wrap) mag = -(mag + (float)L);
    return make_float4(s[0], s[1], s[2], mag);
}

// MODE 0: count the pairs of every leaf; 1: fill the CSR rows (row from a
// scan of the counts); 2: count and fill fixed rows of `cap` entries at
// I * cap (a row that does not fit sets *overflow; the host then walks again
// in modes 0 and 1).
template <int MODE>
__global__ void pair_walk_k(Nodes nd, Leaves lv, const BoxDev *__restrict__ boxes, int nleaf,
                            int hydro, uint32_t *counts, const uint32_t *__restrict__ row,
                            uint32_t *col, float4 *frame, uint32_t *start, uint32_t cap, uint32_t *overflow,
                            const uint8_t *__restrict__ mask, const uint32_t *nl_dev)
{
    constexpr bool FILL = MODE != 0;
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nleaf) return;
    if (I >= leaves_of(nleaf, nl_dev)) {
        if (MODE != 1) counts[I] = 0;
        return;
    }
    // leaves without a row: DM leaves of the hydro list, unmasked leaves
    if ((hydro && lv.species[I] != CRK_GAS) || (mask && !mask[I])) {
        if (MODE != 1) counts[I] = 0;
        return;
    }
    const int32_t slot = (int32_t)lv.slot[I];
    const BoxDev bx = boxes[slot];
    const float L = (float)bx.L, hL = 0.5f * L;
    const float4 ilo = nd.lo[I], ihi = nd.hi[I];
    const float cix = 0.5f * (ilo.x + ihi.x), ciy = 0.5f * (ilo.y + ihi.y), ciz = 0.5f * (ilo.z + ihi.z);
    const float eix = 0.5f * (ihi.x - ilo.x), eiy = 0.5f * (ihi.y - ilo.y), eiz = 0.5f * (ihi.z - ilo.z);
    const float RI = hydro ? lv.hmax[I] : (float)bx.r_cut;
    const size_t base = MODE == 1 ? (size_t)row[I] : MODE == 2 ? (size_t)I * cap : 0u;
    uint32_t cnt = 0;
    // stack entries: level << 26 | index within the level (nleaf < 2^26)
    uint32_t stack[96];
    int sp = 0;
    stack[sp++] = (uint32_t)(nd.levels - 1) << 26;
    while (sp > 0) {
        const uint32_t e = stack[--sp];
        const int l = (int)(e >> 26), k = (int)(e & 0x3ffffffu);
        const int64_t off = nd.level_off[l] + k;
        const float4 nlo = nd.lo[off], nhi = nd.hi[off];
        const int32_t ns = __float_as_int(nhi.w);
        if (ns != -1 && ns != slot) continue;
        const float nh = nlo.w;
        if (hydro && !(nh > 0.f)) continue;
        if (ns == slot) {
            const float R = hydro ? fmaxf(RI, nh) : RI;
            const float Rm = R * 1.0001f + 1e-5f * L;
            float gap2 = 0.f;
            float d, g;
            d = 0.5f * (nlo.x + nhi.x) - cix;
            if (d >= hL) d -= L; else if (d < -hL) d += L;
            // extents summed first: the test is exactly symmetric in (I, J)
            g = fabsf(d) - (eix + 0.5f * (nhi.x - nlo.x));
            if (g > 0.f) gap2 += g * g;
            d = 0.5f * (nlo.y + nhi.y) - ciy;
            if (d >= hL) d -= L; else if (d < -hL) d += L;
            g = fabsf(d) - (eiy + 0.5f * (nhi.y - nlo.y));
            if (g > 0.f) gap2 += g * g;
            d = 0.5f * (nlo.z + nhi.z) - ciz;
            if (d >= hL) d -= L; else if (d < -hL) d += L;
            g = fabsf(d) - (eiz + 0.5f * (nhi.z - nlo.z));
            if (g > 0.f) gap2 += g * g;
            if (gap2 >= Rm * Rm) continue;
        }
        if (l == 0) {
            if (FILL && (MODE == 1 || cnt < cap)) {
                col[base + cnt] = (uint32_t)k;
                frame[base + cnt] = pair_frame(lv, I, k, bx.L);
                if (start) start[base + cnt] = lv.start[k];
            }
            ++cnt;
        } else {
            const int64_t nchild = nd.level_off[l] - nd.level_off[l - 1];
            const uint32_t lc = (uint32_t)(l - 1) << 26;
            if ((int64_t)2 * k + 1 < nchild) stack[sp++] = lc | (uint32_t)(2 * k + 1);
            stack[sp++] = lc | (uint32_t)(2 * k);
        }
    }
    if (MODE != 1) counts[I] = cnt;
    if (MODE == 2 && cnt > cap) atomicOr(overflow, 1u);
}

// The fixed rows of mode 2 packed into CSR rows; one warp per leaf.
__global__ void pair_compact_k(int nleaf, uint32_t cap, const uint32_t *__restrict__ counts,
                               const uint32_t *__restrict__ row, const uint32_t *__restrict__ scol,
                               const float4 *__restrict__ sframe, const uint32_t *__restrict__ sstart,
                               uint32_t *col, float4 *frame, uint32_t *start, const uint32_t *nl_dev)
{
    const int I = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const uint32_t lane = lane_id();
    if (I >= leaves_of(nleaf, nl_dev)) return;
    const uint32_t c = counts[I], r = row[I];
    const size_t b = (size_t)I * cap;
    for (uint32_t t = lane; t < c; t += 32u) {
        col[r + t] = scol[b + t];
        frame[r + t] = sframe[b + t];
        if (start) start[r + t] = sstart[b + t];
    }
}

// Orders the particles of every leaf so that each run of 32 (the chunks and
// warp target groups of the pair passes) is a compact slab: a leaf's range is
// cut at a multiple of 32 by a plane normal to its longest axis (particles
// ranked by that coordinate, ties by position), then each side again, down to
// 32 (k-d splits inside the base leaf).  perm maps sorted position -> original
// index and is rewritten within each leaf.  One warp per leaf, leaf <= 128.
constexpr int kKdWarps = 4;

struct KdScratch {
    float x[128], y[128], z[128];
    uint32_t id[128];
    float tx[128], ty[128], tz[128];
    uint32_t tid[128];
};

__device__ void kd_sort_range(KdScratch &S, uint32_t lo, uint32_t hi, uint32_t lane)
{
    float mn[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, mx[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    for (uint32_t t = lo + lane; t < hi; t += 32) {
        const float p[3] = {S.x[t], S.y[t], S.z[t]};
#pragma unroll
        for (int a = 0; a < 3; ++a) { mn[a] = fminf(mn[a], p[a]); mx[a] = fmaxf(mx[a], p[a]); }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mn[a] = fminf(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
            mx[a] = fmaxf(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
        }
    int axis = 0;
    if (mx[1] - mn[1] > mx[axis] - mn[axis]) axis = 1;
    if (mx[2] - mn[2] > mx[axis] - mn[axis]) axis = 2;
    const float *key = axis == 0 ? S.x : (axis == 1 ? S.y : S.z);
    for (uint32_t t = lo + lane; t < hi; t += 32) {
        const float kt = key[t];
        uint32_t r = 0;
        for (uint32_t q = lo; q < hi; ++q) {
            const float kq = key[q];
            r += (kq < kt || (kq == kt && q < t)) ? 1u : 0u;
        }
        const uint32_t d = lo + r;
        S.tx[d] = S.x[t];
        S.ty[d] = S.y[t];
        S.tz[d] = S.z[t];
        S.tid[d] = S.id[t];
    }
    __syncwarp();
    for (uint32_t t = lo + lane; t < hi; t += 32) {
        S.x[t] = S.tx[t];
        S.y[t] = S.ty[t];
        S.z[t] = S.tz[t];
        S.id[t] = S.tid[t];
    }
    __syncwarp();
}

__global__ void kd_order_k(State s, Leaves lv, int nleaf, uint32_t *perm, const uint32_t *nl_dev)
{
    __shared__ KdScratch scratch[kKdWarps];
    const uint32_t w = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    const int L = blockIdx.x * kKdWarps + (int)w;
    if (L >= leaves_of(nleaf, nl_dev)) return;
    const uint32_t s0 = lv.start[L], c = lv.count[L];
    if (c <= 1u) return;
    KdScratch &S = scratch[w];
    const uint32_t id0 = perm[s0];
    const double x0 = s.x[id0], y0 = s.y[id0], z0 = s.z[id0];
    for (uint32_t t = lane; t < c; t += 32) {
        const uint32_t id = perm[s0 + t];
        S.x[t] = (float)(s.x[id] - x0);
        S.y[t] = (float)(s.y[id] - y0);
        S.z[t] = (float)(s.z[id] - z0);
        S.id[t] = id;
    }
    __syncwarp();
    const uint32_t g = (c + 31u) / 32u;
    // every leaf is ordered, small ones too: the order inside a leaf is then a
    // function of its particles' positions alone, whatever order the sort
    // left them in (it orders only the key bits the leaves need)
    kd_sort_range(S, 0, c, lane);
    const uint32_t cut = 32u * ((g + 1u) / 2u);
    if (cut > 32u) kd_sort_range(S, 0, cut, lane);
    if (c > cut + 32u) kd_sort_range(S, cut, c, lane);
    for (uint32_t t = lane; t < c; t += 32) perm[s0 + t] = S.id[t];
}

// Warp work items of the pair passes: every leaf is cut into target groups
// of at most 32 consecutive particles; (leaf, first particle offset).
__global__ void group_count_k(Leaves lv, int nleaf, int gas_only, uint32_t *counts, const uint32_t *nl_dev)
{
    const int L = blockIdx.x * blockDim.x + threadIdx.x;
    if (L >= nleaf) return;
    if (L >= leaves_of(nleaf, nl_dev)) {
        counts[L] = 0u;
        return;
    }
    counts[L] = (gas_only && lv.species[L] != CRK_GAS) ? 0u : (lv.count[L] + 31u) / 32u;
}

__global__ void group_fill_k(Leaves lv, int nleaf, int gas_only, const uint32_t *__restrict__ off,
                             uint2 *groups, const uint32_t *nl_dev)
{
    const int L = blockIdx.x * blockDim.x + threadIdx.x;
    if (L >= leaves_of(nleaf, nl_dev)) return;
    if (gas_only && lv.species[L] != CRK_GAS) return;
    const uint32_t ng = (lv.count[L] + 31u) / 32u;
    for (uint32_t g = 0; g < ng; ++g) groups[off[L] + g] = make_uint2((uint32_t)L, 32u * g);
}

inline unsigned grid_for(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

void launch_leaf_kd_order(const State &unsorted, const Leaves &lv, int nleaf, uint32_t *perm, cudaStream_t st,
                          const uint32_t *nl_dev)
{
    if (nleaf <= 0) return;
    kd_order_k<<<grid_for(nleaf, kKdWarps), 32 * kKdWarps, 0, st>>>(unsorted, lv, nleaf, perm, nl_dev);
    note_launches(1);
}

void launch_group_count(const Leaves &lv, int nleaf, int gas_only, uint32_t *counts, cudaStream_t st,
                        const uint32_t *nl_dev)
{
    if (nleaf <= 0) return;
    group_count_k<<<grid_for(nleaf, kT), kT, 0, st>>>(lv, nleaf, gas_only, counts, nl_dev);
    note_launches(1);
}

void launch_group_fill(const Leaves &lv, int nleaf, int gas_only, const uint32_t *off, uint2 *groups,
                       cudaStream_t st, const uint32_t *nl_dev)
{
    if (nleaf <= 0) return;
    group_fill_k<<<grid_for(nleaf, kT), kT, 0, st>>>(lv, nleaf, gas_only, off, groups, nl_dev);
    note_launches(1);
}

size_t scan_tmp_words(int64_t n) { return scan_tmp_words_for(n); }

void scan_exclusive_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *total,
                        uint32_t *tmp, cudaStream_t st)
{
    if (n <= 0) {
        if (total) cudaMemsetAsync(total, 0, sizeof(uint32_t), st);
        return;
    }
    int64_t nb = (n + kTile - 1) / kTile;
    scan_reduce_k<<<(unsigned)nb, kT, 0, st>>>(in, n, tmp);
    scan_partials_k<<<1, 1024, 0, st>>>(tmp, nb, total);
    scan_down_k<<<(unsigned)nb, kT, 0, st>>>(in, out, n, tmp);
    note_launches(3);
}

size_t radix_count_words(int64_t n) { return radix_count_words_for(n); }

void radix_sort_u64(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt,
                    int64_t n, uint32_t *counts, uint32_t *scan_tmp, int first_bit, int end_bit,
                    cudaStream_t st, uint64_t **keys_out, uint32_t **vals_out)
{
    uint64_t *ki = keys, *ko = keys_alt;
    uint32_t *vi = vals, *vo = vals_alt;
    if (n > 0) {
        int64_t nb = (n + kTile - 1) / kTile;
        for (int shift = first_bit; shift < end_bit; shift += 8) {
            radix_hist_k<<<(unsigned)nb, kT, 0, st>>>(ki, n, shift, counts, nb);
            scan_exclusive_u32(counts, counts, 256 * nb, nullptr, scan_tmp, st);
            radix_scatter_k<<<(unsigned)nb, kT, 0, st>>>(ki, vi, ko, vo, n, shift, counts, nb);
            note_launches(2);
            uint64_t *tk = ki; ki = ko; ko = tk;
            uint32_t *tv = vi; vi = vo; vo = tv;
        }
    }
    *keys_out = ki;
    *vals_out = vi;
}

void launch_morton_keys(const State &s, const BoxDev *boxes, int64_t n, int slot_bits,
                        uint64_t *keys, uint32_t *idx, cudaStream_t st)
{
    if (n <= 0) return;
    morton_keys_k<<<grid_for(n, kT), kT, 0, st>>>(s, boxes, n, slot_bits, keys, idx);
    note_launches(1);
}

void launch_permute(const State &src, const State &dst, const uint32_t *perm, int64_t n,
                    cudaStream_t st)
{
    if (n <= 0) return;
    permute_k<<<grid_for(n, kT), kT, 0, st>>>(src, dst, perm, n);
    note_launches(1);
}

void launch_leaf_flags(const uint64_t *keys, int slot_bits, const BoxDev *boxes, int64_t n,
                       int cap, uint32_t *flags, int first_bit, uint32_t *stats, cudaStream_t st)
{
    if (n <= 0) return;
    leaf_flags_k<<<grid_for(n, kT), kT, 0, st>>>(keys, slot_bits, boxes, n, cap, flags, first_bit, stats);
    note_launches(1);
}

void launch_leaf_setup(const uint32_t *flags, const uint32_t *scan, int64_t n, int nleaf,
                       Leaves lv, cudaStream_t st, const uint32_t *nl_dev)
{
    if (n <= 0 || nleaf <= 0) return;
    leaf_setup_k<<<grid_for(n, kT), kT, 0, st>>>(flags, scan, n, (uint32_t)nleaf, lv.start);
    leaf_count_k<<<grid_for(nleaf, kT), kT, 0, st>>>(lv, nleaf, n, nl_dev);
    note_launches(2);
}

void launch_leaf_bounds(const State &s, const BoxDev *boxes, Leaves lv, int nleaf, int mixed,
                        void *pm, Nodes nd, cudaStream_t st, const uint32_t *nl_dev)
{
    if (nleaf <= 0) return;
    unsigned g = grid_for((int64_t)nleaf * 32, kT);
    if (mixed) leaf_bounds_k<1><<<g, kT, 0, st>>>(s, boxes, lv, nleaf, pm, nd, nl_dev);
    else leaf_bounds_k<0><<<g, kT, 0, st>>>(s, boxes, lv, nleaf, pm, nd, nl_dev);
    note_launches(1);
}

void launch_build_nodes(Nodes &nd, int nleaf, cudaStream_t st)
{
    int64_t cnt = nleaf;
    int l = 0;
    nd.level_off[0] = 0;
    while (cnt > 1) {
        const int64_t np = (cnt + 1) / 2;
        nd.level_off[l + 1] = nd.level_off[l] + cnt;
        node_level_k<<<grid_for(np, kT), kT, 0, st>>>(nd, nd.level_off[l], cnt, nd.level_off[l + 1], np);
        note_launches(1);
        cnt = np;
        ++l;
    }
    nd.level_off[l + 1] = nd.level_off[l] + cnt;
    nd.levels = l + 1;
    nd.total = nd.level_off[l + 1];
}

void launch_pair_count(const Nodes &nd, const Leaves &lv, const BoxDev *boxes, int nleaf,
                       int hydro, uint32_t *counts, cudaStream_t st, const uint8_t *mask, const uint32_t *nl_dev)
{
    if (nleaf <= 0) return;
    pair_walk_k<0><<<grid_for(nleaf, 128), 128, 0, st>>>(nd, lv, boxes, nleaf, hydro, counts,
                                                           nullptr, nullptr, nullptr, nullptr, 0u, nullptr, mask,
                                                           nl_dev);
    note_launches(1);
}

void launch_pair_scratch(const Nodes &nd, const Leaves &lv, const BoxDev *boxes, int nleaf, int hydro,
                         uint32_t *counts, uint32_t cap, uint32_t *col, float4 *frame, uint32_t *start,
                         uint32_t *overflow, cudaStream_t st, const uint8_t *mask, const uint32_t *nl_dev)
{
    if (nleaf <= 0) return;
    pair_walk_k<2><<<grid_for(nleaf, 128), 128, 0, st>>>(nd, lv, boxes, nleaf, hydro, counts, nullptr, col,
                                                           frame, start, cap, overflow, mask, nl_dev);
    note_launches(1);
}

void launch_pair_compact(int nleaf, uint32_t cap, const uint32_t *counts, const uint32_t *row,
                         const uint32_t *scol, const float4 *sframe, const uint32_t *sstart, uint32_t *col,
                         float4 *frame, uint32_t *start, cudaStream_t st, const uint32_t *nl_dev)
{
    if (nleaf <= 0) return;
    pair_compact_k<<<grid_for((int64_t)nleaf * 32, kT), kT, 0, st>>>(nleaf, cap, counts, row, scol, sframe,
                                                                     sstart, col, frame, start, nl_dev);
    note_launches(1);
}

void launch_pair_fill(const Nodes &nd, const Leaves &lv, const BoxDev *boxes, int nleaf,
                      int hydro, const uint32_t *row, uint32_t *col, float4 *frame, uint32_t *start,
                      cudaStream_t st, const uint8_t *mask, const uint32_t *nl_dev)
{
    if (nleaf <= 0) return;
    pair_walk_k<1><<<grid_for(nleaf, 128), 128, 0, st>>>(nd, lv, boxes, nleaf, hydro, nullptr,
                                                           row, col, frame, start, 0u, nullptr, mask, nl_dev);
    note_launches(1);
}

}  // namespace crk
