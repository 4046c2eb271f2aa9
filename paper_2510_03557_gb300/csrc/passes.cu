// The leaf-to-leaf pair passes of the short-range solver (paper Sec. IV-B2,
// Eq. 1-2): density D, kernel moments M fused with the correction solve C,
// the CRKSPH hydro rates H, and short-range gravity G.
//
// Work decomposition: every leaf is cut into target groups of at most 32
// particles; each warp takes one group (lane = target particle i) and runs
// on its own, without block-wide barriers.  For every neighbour leaf J of the
// target leaf's pair list the warp
//   0. skips J when J's box, or one of its 32-particle chunk boxes, is out
//      of range of the warp's own target box,
//   1. stages in warp-private shared memory the records of J's particles
//      that lie in range of the warp's target box, compacted by a ballot
//      (one candidate per lane; the tile is padded with far-away sentinels
//      to a multiple of 32, so the test needs no bounds check),
//   2. tests the staged candidates with a fully unrolled, branch-free loop
//      into a bitmask (about ten instructions per candidate), and
//   3. evaluates the pair function of Eq. 1 on the set bits only,
// accumulating phi_i in registers.  No atomics and a fixed order: results are
// deterministic, and a box gives bit-identical results alone or batched.
//
// Two arithmetic forms share the code:
//   mixed  (R = float):  positions are FP32 offsets from each leaf's FP64
//          centre; the leaf-pair shift wrap(c_J - c_I) comes with the pair
//          list (formed in FP64 once per pair), so FP32 differences stay
//          small.  Neighbour-set membership that decides an integer (counts,
//          hashes) or a discontinuous force (the gravity cut) is re-decided
//          in FP64, with the exact expression of the definition, whenever the
//          FP32 r^2 lies in a guard band around the threshold that bounds its
//          rounding error.  Square roots, reciprocals and quotients use the
//          hardware approximations.
//   plain  (R = double): absolute FP64 positions, the same minimum-image and
//          r^2 expression (no FMA) as the definition, every operation FP64.
#include "crk_internal.h"

#include <cfloat>

namespace crk {

namespace {

constexpr int kWarps = 4;             // warps (target groups) per CTA
// Resident CTAs per SM the mixed form's pass kernels are compiled for (a
// register budget: 65,536 / (128 x blocks) per thread; 0 = no bound)
constexpr int kMomentsMinBlocks = 5;
constexpr int kHydroMinBlocks = 4;
constexpr int kFillMinBlocks = 0;
constexpr int kBlock = 32 * kWarps;

constexpr double kPi = 3.14159265358979323846;
// Wendland C4 in 3-D with support H = 2h:
//   W = kWn / H^3 (1-q)^6 (1 + 6q + 35 q^2 / 3),  q = r / H
//   grad_i W = g x_ij,  g = -(56/3) kWn / H^5 (1 + 5q)(1-q)^5
constexpr double kWn = 495.0 / (32.0 * kPi);
constexpr double kGn = -(56.0 / 3.0) * kWn;
// Abramowitz & Stegun 7.1.26 (Hastings): erfc(x) ~ t P(t) exp(-x^2),
// t = 1/(1 + p x), |error| <= 1.5e-7 for x >= 0.
constexpr float kAsP = 0.3275911f;
constexpr float kLog2e = 1.44269504088896341f;  // log2(e)
// The mixed gravity factor in v = u sqrt(log2 e), so that exp(-u^2) = 2^(-v^2):
// 1 + p u = 1 + (p / sqrt(log2 e)) v and 2u / sqrt(pi) = (2 / (sqrt(pi) sqrt(log2 e))) v.
constexpr double kSqrtLog2e = 1.20112240878644981;
constexpr float kAsPv = (float)(0.3275911 / kSqrtLog2e);
constexpr float kTwoOverSqrtPiV = (float)(1.12837916709551257390 / kSqrtLog2e);
constexpr float kAs1 = 0.254829592f, kAs2 = -0.284496736f, kAs3 = 1.421413741f,
                kAs4 = -1.453152027f, kAs5 = 1.061405429f;
constexpr double kTwoOverSqrtPi = 1.12837916709551257390;
constexpr float kEps32 = 5.9604645e-8f;  // 2^-24

template <typename R> struct Real;
template <> struct Real<float> {
    static constexpr bool mixed = true;
    static constexpr float far = 1e30f;  // sentinel coordinate: r^2 overflows to +inf
    __device__ static float sqrt_(float x)
    {
        float y;
        asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    }
    __device__ static float rcp(float x)
    {
        float y;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    }
    __device__ static float rsqrt(float x)
    {
        float y;
        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    }
    // 2^x by the hardware approximation (inputs and results here are normal)
    __device__ static float exp2(float x)
    {
        float y;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    }
    __device__ static float log2(float x)
    {
        float y;
        asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    }
    __device__ static float div(float a, float b) { return __fdividef(a, b); }
    __device__ static float r2(float dx, float dy, float dz) { return fmaf(dz, dz, fmaf(dy, dy, dx * dx)); }
    __device__ static float mul_rn(float a, float b) { return __fmul_rn(a, b); }
    __device__ static float add_rn(float a, float b) { return __fadd_rn(a, b); }
};
template <> struct Real<double> {
    static constexpr bool mixed = false;
    static constexpr double far = 1e300;
    __device__ static double sqrt_(double x) { return sqrt(x); }
    __device__ static double rcp(double x) { return 1.0 / x; }
    __device__ static double div(double a, double b) { return a / b; }
    // (dx*dx + dy*dy) + dz*dz with every product and sum rounded on its own,
    // as the neighbour predicate is defined.
    __device__ static double r2(double dx, double dy, double dz)
    {
        return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    }
    __device__ static double mul_rn(double a, double b) { return __dmul_rn(a, b); }
    __device__ static double add_rn(double a, double b) { return __dadd_rn(a, b); }
};

template <typename R>
__device__ __forceinline__ R wrap1(R d, R L, R hL)
{
    if (d >= hL) d -= L;
    else if (d < -hL) d += L;
    return d;
}

__device__ __forceinline__ uint64_t mix64(uint64_t x)
{
    // SplitMix64 output function (Steele, Lea & Flood 2014).
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ float warp_min(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// The neighbour predicate exactly as defined: FP64 positions, one wrap,
// (dx*dx + dy*dy) + dz*dz without contraction, strict comparison.
__device__ __forceinline__ bool exact_lt(const State &s, uint32_t i, uint32_t j, double L,
                                         double thr2)
{
    const double hL = 0.5 * L;
    double dx = wrap1(s.x[j] - s.x[i], L, hL);
    double dy = wrap1(s.y[j] - s.y[i], L, hL);
    double dz = wrap1(s.z[j] - s.z[i], L, hL);
    return Real<double>::r2(dx, dy, dz) < thr2;
}

// Guard band of the mixed form around a squared threshold T^2: the FP32 r^2
// differs from the exact one by less than 8 sqrt(3) eps T mag + 3 eps T^2
// (four roundings per coordinate difference, three in the sum of squares);
// the band is several times wider and never below 1e-5 T^2.
__device__ __forceinline__ float guard_band(float T, float mag)
{
    return 1e-5f * T * T + 64.0f * kEps32 * T * (mag + T);
}

// Box of the warp's targets relative to the target leaf's centre.
struct WarpBox {
    float cx, cy, cz, ex, ey, ez;
};

__device__ __forceinline__ WarpBox warp_box(float px, float py, float pz, bool act)
{
    const float lx = warp_min(act ? px : FLT_MAX), hx = warp_max(act ? px : -FLT_MAX);
    const float ly = warp_min(act ? py : FLT_MAX), hy = warp_max(act ? py : -FLT_MAX);
    const float lz = warp_min(act ? pz : FLT_MAX), hz = warp_max(act ? pz : -FLT_MAX);
    WarpBox b;
    b.cx = 0.5f * (lx + hx); b.cy = 0.5f * (ly + hy); b.cz = 0.5f * (lz + hz);
    b.ex = 0.5f * (hx - lx); b.ey = 0.5f * (hy - ly); b.ez = 0.5f * (hz - lz);
    return b;
}

// True when leaf J (box [s - e_J, s + e_J] in the target leaf's frame, from
// the pair frame fr) lies at distance >= R from the warp's target box.  Pairs
// that still need a per-pair wrap (fr.w < 0) are never skipped.
__device__ __forceinline__ bool out_of_range(const WarpBox &b, const float4 &fr, float ex, float ey,
                                             float ez, float R)
{
    if (fr.w < 0.f) return false;
    float gap2 = 0.f, g;
    g = fabsf(fr.x - b.cx) - ex - b.ex;
    if (g > 0.f) gap2 += g * g;
    g = fabsf(fr.y - b.cy) - ey - b.ey;
    if (g > 0.f) gap2 += g * g;
    g = fabsf(fr.z - b.cz) - ez - b.ez;
    if (g > 0.f) gap2 += g * g;
    return gap2 >= R * R;
}

// Mask of leaf J's 32-particle chunks whose boxes (J's frame) lie within R of
// the warp's target box (shifted into J's frame by -s).  All of J's chunks
// when a per-pair wrap is needed.
__device__ __forceinline__ uint32_t chunks_in_range(const Leaves &lv, uint32_t J, uint32_t cJ,
                                                    const WarpBox &b, const float4 &fr, float R)
{
    const uint32_t nch = (cJ + 31u) / 32u;
    if (fr.w < 0.f) return (1u << nch) - 1u;
    const float cx = b.cx - fr.x, cy = b.cy - fr.y, cz = b.cz - fr.z;
    uint32_t mask = 0;
#pragma unroll
    for (int c = 0; c < kChunks; ++c) {
        if ((uint32_t)c >= nch) break;
        const float4 lo = lv.clo[(size_t)J * kChunks + c], hi = lv.chi[(size_t)J * kChunks + c];
        float gap2 = 0.f, g;
        g = fabsf(0.5f * (lo.x + hi.x) - cx) - 0.5f * (hi.x - lo.x) - b.ex;
        if (g > 0.f) gap2 += g * g;
        g = fabsf(0.5f * (lo.y + hi.y) - cy) - 0.5f * (hi.y - lo.y) - b.ey;
        if (g > 0.f) gap2 += g * g;
        g = fabsf(0.5f * (lo.z + hi.z) - cz) - 0.5f * (hi.z - lo.z) - b.ez;
        if (g > 0.f) gap2 += g * g;
        if (gap2 < R * R) mask |= 1u << c;
    }
    return mask;
}

// Target position q in the frame of the staged leaf J.
template <typename R>
struct Target {
    R qx, qy, qz;
    bool wrap;
    float mag;
};

template <typename R>
__device__ __forceinline__ Target<R> target_in_frame(const Vec4<R> &ri, const float4 &fr)
{
    Target<R> q;
    if (Real<R>::mixed) {
        q.qx = ri.x - (R)fr.x;
        q.qy = ri.y - (R)fr.y;
        q.qz = ri.z - (R)fr.z;
        q.wrap = fr.w < 0.f;
        q.mag = fabsf(fr.w);
    } else {
        q.qx = ri.x;
        q.qy = ri.y;
        q.qz = ri.z;
        q.wrap = true;
        q.mag = 0.f;
    }
    return q;
}

// r^2 and x_j - x_i for a staged record.
template <typename R, bool WRAP>
__device__ __forceinline__ R sep2(const Vec4<R> &rj, const Target<R> &q, R L, R hL, R &dx, R &dy, R &dz)
{
    dx = rj.x - q.qx;
    dy = rj.y - q.qy;
    dz = rj.z - q.qz;
    if (WRAP) {
        dx = wrap1(dx, L, hL);
        dy = wrap1(dy, L, hL);
        dz = wrap1(dz, L, hL);
    }
    return Real<R>::r2(dx, dy, dz);
}

// Candidate test over a staged tile: bit j of m[j/32] set when r^2 < thr
// (one threshold per target) or r^2 < max(thr, thrj[j]) (per candidate).
// Only the 32-slot chunks set in cm are staged and tested.
template <typename R, int JMAX, bool WRAP, bool PERJ>
__device__ __forceinline__ void test_tile(const Vec4<R> *tile, const float *thrj, const Target<R> &q,
                                          R L, R hL, R thr, uint32_t cm, uint32_t (&m)[JMAX / 32])
{
#pragma unroll
    for (int w = 0; w < JMAX / 32; ++w) {
        uint32_t bits = 0;
        m[w] = 0;
        if (!((cm >> w) & 1u)) continue;
#pragma unroll 8
        for (int b = 0; b < 32; ++b) {
            const int j = 32 * w + b;
            R dx, dy, dz;
            const R r2 = sep2<R, WRAP>(tile[j], q, L, hL, dx, dy, dz);
            R t = thr;
            if (PERJ) t = fmax(thr, (R)thrj[j]);
            bits |= (r2 < t ? 1u : 0u) << b;
        }
        m[w] = bits;
    }
}

template <typename R, int JMAX, bool PERJ>
__device__ __forceinline__ void test_tile_any(const Vec4<R> *tile, const float *thrj,
                                              const Target<R> &q, R L, R hL, R thr, uint32_t cm,
                                              uint32_t (&m)[JMAX / 32])
{
    if (q.wrap) test_tile<R, JMAX, true, PERJ>(tile, thrj, q, L, hL, thr, cm, m);
    else test_tile<R, JMAX, false, PERJ>(tile, thrj, q, L, hL, thr, cm, m);
}

// The hydro union test over a staged tile in one sweep: bit j of mu[j/32]
// when r^2 < max(thr, thrj[j]) (r < H_i or r < H_j), bit j of mg[j/32] when
// r^2 < thr (the gather set r < H_i).
template <typename R, int JMAX, bool WRAP>
__device__ __forceinline__ void test_tile_union(const Vec4<R> *tile, const float *thrj, const Target<R> &q, R L,
                                                R hL, R thr, uint32_t cm, uint32_t (&mu)[JMAX / 32],
                                                uint32_t (&mg)[JMAX / 32])
{
#pragma unroll
    for (int w = 0; w < JMAX / 32; ++w) {
        uint32_t bu = 0, bg = 0;
        mu[w] = 0;
        mg[w] = 0;
        if (!((cm >> w) & 1u)) continue;
#pragma unroll 8
        for (int b = 0; b < 32; ++b) {
            const int j = 32 * w + b;
            R dx, dy, dz;
            const R r2 = sep2<R, WRAP>(tile[j], q, L, hL, dx, dy, dz);
            bu |= (r2 < fmax(thr, (R)thrj[j]) ? 1u : 0u) << b;
            bg |= (r2 < thr ? 1u : 0u) << b;
        }
        mu[w] = bu;
        mg[w] = bg;
    }
}

template <typename R>
__device__ __forceinline__ void kernel_wg(R r, R invH, R cW, R cG, R &W, R &g)
{
    const R q = r * invH;
    R om = (R)1 - q;
    om = om > (R)0 ? om : (R)0;
    const R om2 = om * om;
    const R om4 = om2 * om2;
    const R om5 = om4 * om;
    W = cW * om5 * om * ((R)1 + q * ((R)6 + q * (R)(35.0 / 3.0)));
    g = cG * om5 * ((R)1 + (R)5 * q);
}

__device__ __forceinline__ void set_error(int *err, int code, uint32_t id)
{
    atomicCAS(err, 0, code);
    atomicMin(err + 1, (int)id);
}

// Where a staged candidate sits relative to the target leaf's centre, in
// FP32, for the per-candidate cut: mixed records are relative to their own
// leaf's centre and move by the pair frame; FP64 records are absolute.
struct CandFrame {
    float fx, fy, fz;          // mixed: pair frame (c_J - c_I)
    double cx, cy, cz, L, hL;  // FP64: target leaf centre and box
    bool cull;                 // false: keep every candidate (pair needs per-pair wrap)
};

template <typename R>
__device__ __forceinline__ void cand_pos(const Vec4<R> &v, const CandFrame &f, float &x, float &y, float &z)
{
    if (Real<R>::mixed) {
        x = (float)v.x + f.fx;
        y = (float)v.y + f.fy;
        z = (float)v.z + f.fz;
    } else {
        x = (float)wrap1((double)v.x - f.cx, f.L, f.hL);
        y = (float)wrap1((double)v.y - f.cy, f.L, f.hL);
        z = (float)wrap1((double)v.z - f.cz, f.L, f.hL);
    }
}

template <typename R>
__device__ __forceinline__ CandFrame cand_frame(const Leaves &lv, int I, const float4 &fr, double L)
{
    CandFrame f;
    f.fx = fr.x;
    f.fy = fr.y;
    f.fz = fr.z;
    f.cx = lv.cx[I];
    f.cy = lv.cy[I];
    f.cz = lv.cz[I];
    f.L = L;
    f.hL = 0.5 * L;
    // one wrap of (x_j - c_I) is exact only when no two points of the two
    // leaves are L/2 apart on an axis, which the frame's sign certifies
    f.cull = fr.w >= 0.f;
    return f;
}

// Greatest common divisor (Euclid).
__device__ __forceinline__ uint32_t gcd_u32(uint32_t a, uint32_t b)
{
    while (b) {
        const uint32_t r = a % b;
        a = b;
        b = r;
    }
    return a;
}

__device__ __forceinline__ float box_gap2(const WarpBox &b, float x, float y, float z)
{
    float gap2 = 0.f, g;
    g = fabsf(x - b.cx) - b.ex;
    if (g > 0.f) gap2 += g * g;
    g = fabsf(y - b.cy) - b.ey;
    if (g > 0.f) gap2 += g * g;
    g = fabsf(z - b.cz) - b.ez;
    if (g > 0.f) gap2 += g * g;
    return gap2;
}

// Stages, compacted in J's order, the candidates of leaf J that can reach
// the warp's target box: candidate k < cJ (in a 32-chunk set in cm) is kept
// when its distance to the box is below Rc, or below its own radius when
// PERJ (hydro: 2 h_j from hrec1, whose square also goes to h2j).  Writes
// tile[0, K) and slot[0, K) (k of each kept candidate), the record's w
// multiplied by wscale (LOGW: log2 of that), pads the tile to a multiple of 32
// with far-away sentinels (h2j 0), and returns K.
template <typename R, bool PERJ, bool LOGW = false>
__device__ __forceinline__ uint32_t stage_cull(Vec4<R> *tile, uint8_t *slot, float *h2j,
                                               const Vec4<R> *__restrict__ src,
                                               const Vec4<R> *__restrict__ rec1, uint32_t sJ, uint32_t cJ,
                                               uint32_t cm, const WarpBox &wb, const CandFrame &f, float Rc,
                                               uint32_t lane, R wscale = (R)1)
{
    uint32_t K = 0;
    const uint32_t nch = (cJ + 31u) / 32u;
    for (uint32_t c = 0; c < nch; ++c) {
        if (!((cm >> c) & 1u)) continue;
        const uint32_t k = 32u * c + lane;
        bool keep = false;
        Vec4<R> v;
        float Hj2 = 0.f;
        if (k < cJ) {
            v = src[sJ + k];
            float R2 = Rc * Rc;
            if (PERJ) {
                const float Hj = 2.0f * (float)rec1[sJ + k].w;
                Hj2 = Hj * Hj;
                const float Rj = Hj * 1.0001f + 1e-6f * (float)f.L;
                R2 = fmaxf(R2, Rj * Rj);
            }
            keep = true;
            if (f.cull) {
                float x, y, z;
                cand_pos(v, f, x, y, z);
                keep = box_gap2(wb, x, y, z) < R2;
            }
        }
        const uint32_t bal = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            const uint32_t pos = K + __popc(bal & ((1u << lane) - 1u));
            v.w = LOGW ? (R)Real<float>::log2((float)(wscale * v.w)) : wscale * v.w;
            tile[pos] = v;
            slot[pos] = (uint8_t)k;
            if (PERJ) h2j[pos] = Hj2;
        }
        K += __popc(bal);
    }
    const uint32_t end = (K + 31u) & ~31u;
    if (K + lane < end) {
        Vec4<R> s;
        s.x = Real<R>::far;
        s.y = Real<R>::far;
        s.z = Real<R>::far;
        s.w = 0;
        tile[K + lane] = s;
        if (PERJ) h2j[K + lane] = 0.f;
    }
    return K;
}

__device__ __forceinline__ uint32_t chunk_mask(uint32_t K) { return K >= 128u ? 0xfu : (1u << ((K + 31u) / 32u)) - 1u; }

// Work items of a warp pass: groups of up to 32 targets of one leaf.  With
// no queue the launch has one warp per item (n items known on the host).
// With a queue the launch is persistent (a fixed grid filling the SMs): each
// warp takes the next item from a device counter until the item count, read
// on the device, is exhausted, so a pass over every box of a batch needs
// neither the host to know how many items there are nor a launch sized to
// them, and uneven boxes share the SMs item by item.
enum QueueSlot { Q_HCOUNT, Q_HFILL, Q_DONLY, Q_HBOUND, Q_KEEP, Q_DENS, Q_MOM, Q_HYDRO, Q_GRAV, Q_GSYM, Q_N };
static_assert(Q_N <= kQueueSlots, "work-queue slots of the device sizes block");

template <class F>
__device__ __forceinline__ void for_each_item(uint32_t n_host, const uint32_t *n_dev, uint32_t *queue, int slot,
                                              F &&body)
{
    const uint32_t w = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    if (!queue) {
        const uint32_t gi = blockIdx.x * kWarps + w;
        if (gi < (n_dev ? *n_dev : n_host)) body(gi);
        return;
    }
    const uint32_t n = n_dev ? *n_dev : n_host;
    // the next item is taken while the current one runs (its latency hidden)
    uint32_t next = 0;
    if (lane == 0) next = atomicAdd(queue + slot, 1u);
    next = __shfl_sync(0xffffffffu, next, 0);
    while (next < n) {
        const uint32_t gi = next;
        if (lane == 0) next = atomicAdd(queue + slot, 1u);
        body(gi);
        next = __shfl_sync(0xffffffffu, next, 0);
    }
}

// The warp's target group: up to 32 consecutive particles of leaf I.
struct Group {
    int I;
    uint32_t s0, cnt, i;
    bool act;
};

__device__ __forceinline__ Group load_group(const Leaves &lv, const uint2 *groups, uint32_t gi,
                                            uint32_t lane)
{
    const uint2 g = groups[gi];
    Group r;
    r.I = (int)g.x;
    r.s0 = lv.start[r.I] + g.y;
    const uint32_t left = lv.count[r.I] - g.y;
    r.cnt = left < 32u ? left : 32u;
    r.act = lane < r.cnt;
    r.i = r.s0 + (r.act ? lane : 0u);
    return r;
}

// Position of a target relative to its leaf centre, in FP32 (for the warp box).
template <typename R>
__device__ __forceinline__ void rel_pos(const Vec4<R> &ri, const Leaves &lv, int I, double L, float &x,
                                        float &y, float &z)
{
    if (Real<R>::mixed) {
        x = (float)ri.x;
        y = (float)ri.y;
        z = (float)ri.z;
    } else {
        // absolute FP64 records; the leaf centre may lie past a periodic face
        x = (float)wrap1((double)ri.x - lv.cx[I], L, 0.5 * L);
        y = (float)wrap1((double)ri.y - lv.cy[I], L, 0.5 * L);
        z = (float)wrap1((double)ri.z - lv.cz[I], L, 0.5 * L);
    }
}

// ------------------------------------------------------------- records
// Predictor values that enter the forces: v^ = v_half + tau a_old,
// u^ = max(u_half + tau du_old, u_floor) (gas).  hrec1 = (v^, h).  Fixed
// steps: tau = dt/2.  Hierarchical steps, forces at the end of substep s of
// length d: tau = ((s + 1 - s0) - L/2) d for a particle whose steps of L
// substeps started at s0 (dt/2 for the particles whose step ends now).
template <typename R>
__global__ void records_k(PassArgs a)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.n) return;
    const BoxDev &bx = a.boxes[a.s.slot[k]];
    double hdt = bx.hdt;
    if (a.bsub >= 0) {
        const int Lb = 1 << (a.bdepth - (int)a.s.bin[k]);
        const int s0 = (a.bsub / Lb) * Lb;
        hdt = __dmul_rn((double)(2 * (a.bsub + 1 - s0) - Lb), 0.5 * a.bd);
    }
    const double vx = __dadd_rn(a.s.vx[k], __dmul_rn(hdt, a.s.ax[k]));
    const double vy = __dadd_rn(a.s.vy[k], __dmul_rn(hdt, a.s.ay[k]));
    const double vz = __dadd_rn(a.s.vz[k], __dmul_rn(hdt, a.s.az[k]));
    double uh = 0.0;
    if (a.s.species[k] == CRK_GAS) {
        uh = __dadd_rn(a.s.u[k], __dmul_rn(hdt, a.s.du[k]));
        if (uh < bx.u_floor) {
            uh = bx.u_floor;
            if (a.nfloor) atomicAdd(a.nfloor, 1ull);
        }
    }
    Vec4<R> r1;
    r1.x = (R)vx; r1.y = (R)vy; r1.z = (R)vz; r1.w = (R)a.s.h[k];
    reinterpret_cast<Vec4<R> *>(a.hrec[1])[k] = r1;
    reinterpret_cast<R *>(a.uhat)[k] = (R)uh;
}

// Shared memory of one warp: the staged tile and the leaf slot of every
// staged candidate.
template <typename R, int JMAX>
constexpr size_t tile_warp_bytes()
{
    return JMAX * (sizeof(Vec4<R>) + 1);
}

// ------------------------------------------------- hydro neighbour lists
// The density pass tests every candidate pair of the hydro passes once and
// writes, for every gas particle, the list of its hydro neighbours: the
// union set r < H_i or r < H_j, the particle itself included.  Entry k of
// lane l of gas group g sits at row nl_row[g] + k, column l: the lanes of a
// group read one 128-byte row per step.  The fill stages rows in shared
// memory and writes each row once all lanes have passed it.  An entry is one
// 32-bit word: bit 31 set when r < H_i (the gather set of the density and the
// moments), bits 7-30 the position of the leaf pair in row I of the hydro pair
// list (its frame, and the first particle of leaf J in hsj), bits 0-6 the
// neighbour's slot in leaf J.  The moments and hydro passes
// then walk their lists with every lane busy and no candidate test.
constexpr uint32_t kGather = 0x80000000u;
constexpr uint32_t kRowShift = 7;
constexpr uint32_t kMaxRowOffset = 0xffffffu;
constexpr uint32_t kSlotMask = 0x7fu;


template <typename R, int JMAX>
constexpr size_t hlist_warp_bytes()
{
    return JMAX * (sizeof(Vec4<R>) + sizeof(float) + 1);
}

// Rows of list entries a warp of the fill pass holds in shared memory.
constexpr uint32_t kRingRows = 32;
constexpr size_t kRingBytes = kRingRows * 32 * sizeof(uint32_t);

template <typename R, int JMAX>
constexpr size_t hfill_warp_bytes()
{
    return hlist_warp_bytes<R, JMAX>() + kRingBytes;
}

// Entries of the fill pass on their way to global memory: a lane puts entry
// k into ring row k mod kRingRows while k >= base, else writes it directly;
// rows [base, upto) leave as whole 128-byte rows.
struct ListRing {
    uint32_t *rj;
    uint32_t base;
    size_t e0;       // the lane's entry 0 in global memory

    __device__ __forceinline__ void put(const PassArgs &a, uint32_t k, uint32_t lane, uint32_t entry)
    {
        if (k >= base) rj[(k % kRingRows) * 32u + lane] = entry;
        else a.nl_j[e0 + (size_t)k * 32u] = entry;
    }
    // writes rows [base, upto) below cap (the group's rows) whole: a lane's
    // own entries (k: entries it has put) and a filler word where it has
    // none, so that every row leaves as one full 128-byte line (a partly
    // written line costs the L2 a read of it from DRAM when it is evicted)
    __device__ __forceinline__ void flush(const PassArgs &a, uint32_t upto, uint32_t k, uint32_t cap, uint32_t lane)
    {
        const uint32_t end = upto < cap ? upto : cap;
        for (uint32_t r = base; r < end; ++r)
            a.nl_j[e0 + (size_t)r * 32u] = r < k ? rj[(r % kRingRows) * 32u + lane] : 0u;
        base = upto;
    }
};

// Visit order of a leaf-pair row of n entries: entry (t * stride) mod n at
// step t, the stride the smallest odd number >= 7 coprime to n.  The row is in
// Morton order, so consecutive entries lie on one side of the target leaf;
// striding through it spreads every run of visits over all sides, and the
// 32 targets of a warp gain neighbours at similar rates.
struct RowOrder {
    uint32_t n, stride;
    __device__ __forceinline__ explicit RowOrder(uint32_t len) : n(len), stride(7u)
    {
        while (n > 1u && gcd_u32(stride, n) != 1u) stride += 2u;
    }
    __device__ __forceinline__ uint32_t at(uint32_t t) const
    {
        return (uint32_t)(((uint64_t)t * stride) % n);
    }
};

// Target-side thresholds of the hydro neighbour test: r^2 < H_i^2 (plus the
// guard band when the gather set is counted exactly).
template <typename R>
struct HTarget {
    R H, H2, invH, cW;
    double H2x;
};

template <typename R>
__device__ __forceinline__ HTarget<R> hydro_target(const State &s, uint32_t i)
{
    HTarget<R> t;
    const double H64 = 2.0 * s.h[i];
    t.H2x = __dmul_rn(H64, H64);
    t.H = (R)H64;
    // rounded on its own: the count and fill passes must draw the same sets
    t.H2 = Real<R>::mixed ? Real<R>::mul_rn(t.H, t.H) : (R)t.H2x;
    t.invH = Real<R>::rcp(t.H);
    t.cW = (R)kWn * t.invH * t.invH * t.invH;
    return t;
}

// Stages leaf J (row entry p) for the hydro neighbour test of the warp and
// returns the number of staged candidates (0: none in range).
template <typename R, int JMAX>
__device__ __forceinline__ uint32_t hydro_stage(const PassArgs &a, uint32_t p, int I, const WarpBox &wb, float Hw,
                                                double Ld, Vec4<R> *tile, float *h2j, uint8_t *tslot,
                                                uint32_t lane, uint32_t &sJ, float4 &fr)
{
    const uint32_t J = a.hcol[p];
    fr = a.hfr[p];
    const float Rc = fmaxf(Hw, a.lv.hmax[J]) * 1.0001f + 1e-6f * (float)Ld;
    if (out_of_range(wb, fr, a.lv.ex[J], a.lv.ey[J], a.lv.ez[J], Rc)) return 0u;
    sJ = a.lv.start[J];
    const uint32_t cJ = a.lv.count[J];
    const uint32_t cm = chunks_in_range(a.lv, J, cJ, wb, fr, Rc);
    if (cm == 0u) return 0u;
    __syncwarp();
    const uint32_t K = stage_cull<R, true>(tile, tslot, h2j, reinterpret_cast<const Vec4<R> *>(a.pm),
                                           reinterpret_cast<const Vec4<R> *>(a.hrec[1]), sJ, cJ, cm, wb,
                                           cand_frame<R>(a.lv, I, fr, Ld), Hw * 1.0001f + 1e-6f * (float)Ld,
                                           lane);
    __syncwarp();
    return K;
}

// Size of every gas particle's hydro neighbour list, and the largest of
// every group (its number of rows).
template <typename R, int JMAX, bool COUNT>
__global__ void __launch_bounds__(kBlock) hlist_count_k(PassArgs a)
{
    using R4 = Vec4<R>;
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t w = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    for_each_item(a.n_ggas, a.ggas_dev, a.queue, Q_HCOUNT, [&](const uint32_t gi) {
    unsigned char *base = smem + (size_t)w * hlist_warp_bytes<R, JMAX>();
    R4 *tile = reinterpret_cast<R4 *>(base);
    float *h2j = reinterpret_cast<float *>(tile + JMAX);
    uint8_t *tslot = reinterpret_cast<uint8_t *>(h2j + JMAX);
    const Group G = load_group(a.lv, a.ggas, gi, lane);
    const int I = G.I;
    const uint32_t i = G.i;
    const double Ld = a.boxes[a.lv.slot[I]].L;
    const R L = (R)Ld, hL = (R)(0.5 * Ld);
    const R4 ri = reinterpret_cast<const R4 *>(a.pm)[i];
    const HTarget<R> ht = hydro_target<R>(a.s, i);
    float px, py, pz;
    rel_pos(ri, a.lv, I, Ld, px, py, pz);
    const WarpBox wb = warp_box(px, py, pz, G.act);
    const float Hw = warp_max(G.act ? (float)ht.H : 0.f);
    uint32_t cnt = 0;
    const RowOrder order(a.hend[I] - a.hrow[I]);
    for (uint32_t t = 0; t < order.n; ++t) {
        const uint32_t p = a.hrow[I] + order.at(t);
        uint32_t sJ;
        float4 fr;
        const uint32_t K = hydro_stage<R, JMAX>(a, p, I, wb, Hw, Ld, tile, h2j, tslot, lane, sJ, fr);
        if (K == 0u) continue;
        const Target<R> q = target_in_frame(ri, fr);
        const R gb = (COUNT && Real<R>::mixed) ? (R)guard_band((float)ht.H, q.mag) : (R)0;
        uint32_t m[JMAX / 32];
        test_tile_any<R, JMAX, true>(tile, h2j, q, L, hL, Real<R>::add_rn(ht.H2, gb), G.act ? chunk_mask(K) : 0u, m);
#pragma unroll
        for (int ww = 0; ww < JMAX / 32; ++ww) cnt += (uint32_t)__popc(m[ww]);
    }
    const uint32_t len = __reduce_max_sync(0xffffffffu, cnt);
    if (lane == 0) a.nl_len[gi] = len;
    if (G.act) a.nl_cnt[i] = cnt;
    });
}

// V = m/rho, P = (gamma-1) rho u^, c = sqrt(gamma (gamma-1) u^) into the
// hydro records 0 (position, V) and 2 (rho, P, c).
template <typename R>
__device__ __forceinline__ void density_out(const PassArgs &a, uint32_t i, const Vec4<R> &ri, R rho)
{
    const BoxDev &bx = a.boxes[a.s.slot[i]];
    const R uh = reinterpret_cast<const R *>(a.uhat)[i];
    const R gam = (R)bx.gamma;
    const R V = Real<R>::div(ri.w, rho);
    Vec4<R> r0;
    r0.x = ri.x; r0.y = ri.y; r0.z = ri.z; r0.w = V;
    reinterpret_cast<Vec4<R> *>(a.hrec[0])[i] = r0;
    Vec4<R> r2v;
    r2v.x = rho;
    r2v.y = (gam - (R)1) * rho * uh;
    r2v.z = Real<R>::sqrt_(gam * (gam - (R)1) * uh);
    r2v.w = 0;
    reinterpret_cast<Vec4<R> *>(a.hrec[2])[i] = r2v;
}

// Writes every gas particle's hydro neighbour list (the same sets the count
// pass counted, from the same staging and test).
template <typename R, int JMAX, bool COUNT>
__global__ void __launch_bounds__(kBlock, Real<R>::mixed ? kFillMinBlocks : 0) hlist_fill_k(PassArgs a)
{
    using R4 = Vec4<R>;
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t w = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    for_each_item(a.n_ggas, a.ggas_dev, a.queue, Q_HFILL, [&](const uint32_t gi) {
    unsigned char *base = smem + (size_t)w * hfill_warp_bytes<R, JMAX>();
    R4 *tile = reinterpret_cast<R4 *>(base);
    float *h2j = reinterpret_cast<float *>(tile + JMAX);
    uint8_t *tslot = reinterpret_cast<uint8_t *>(h2j + JMAX);
    ListRing ring;
    ring.rj = reinterpret_cast<uint32_t *>(base + hlist_warp_bytes<R, JMAX>());
    ring.base = 0;
    const Group G = load_group(a.lv, a.ggas, gi, lane);
    const int I = G.I;
    const uint32_t i = G.i;
    const double Ld = a.boxes[a.lv.slot[I]].L;
    const R L = (R)Ld, hL = (R)(0.5 * Ld);
    const R4 ri = reinterpret_cast<const R4 *>(a.pm)[i];
    const HTarget<R> ht = hydro_target<R>(a.s, i);
    float px, py, pz;
    rel_pos(ri, a.lv, I, Ld, px, py, pz);
    const WarpBox wb = warp_box(px, py, pz, G.act);
    const float Hw = warp_max(G.act ? (float)ht.H : 0.f);
    ring.e0 = (size_t)a.nl_row[gi] * 32u + lane;
    const uint32_t prow = a.hrow[I];
    // entries the count pass found, or the group's rows when they were sized
    // from the previous step
    const uint32_t room = G.act ? (a.nl_bound ? a.nl_len[gi] : a.nl_cnt[i]) : 0u;
    const uint32_t rows = a.nl_len[gi];  // the group's rows (its longest list, or its bound)
    uint32_t k = 0;
    uint64_t tested = 0;  // staged candidates of the visits (census)
    R rho = 0;  // without neighbour counts the fill pass also forms the density
    const RowOrder order(a.hend[I] - prow);
    for (uint32_t t = 0; t < order.n; ++t) {
        const uint32_t p = prow + order.at(t);
        uint32_t sJ;
        float4 fr;
        const uint32_t K = hydro_stage<R, JMAX>(a, p, I, wb, Hw, Ld, tile, h2j, tslot, lane, sJ, fr);
        if (K == 0u) continue;
        if (COUNT) tested += K;
        const Target<R> q = target_in_frame(ri, fr);
        const R gb = (COUNT && Real<R>::mixed) ? (R)guard_band((float)ht.H, q.mag) : (R)0;
        const R thr = Real<R>::add_rn(ht.H2, gb);
        uint32_t mu[JMAX / 32], mg[JMAX / 32];
        const uint32_t cm = G.act ? chunk_mask(K) : 0u;
        if (q.wrap) test_tile_union<R, JMAX, true>(tile, h2j, q, L, hL, thr, cm, mu, mg);
        else test_tile_union<R, JMAX, false>(tile, h2j, q, L, hL, thr, cm, mu, mg);
        const uint32_t off = p - prow;
        if (off > kMaxRowOffset && lane == 0) set_error(a.err, CRK_EOVERFLOW, a.s.id[i]);
        const uint32_t otag = (off & kMaxRowOffset) << kRowShift;
        uint32_t pop = 0;
#pragma unroll
        for (int ww = 0; ww < JMAX / 32; ++ww) pop += (uint32_t)__popc(mu[ww]);
        // room in the ring for the fastest lane: flush its oldest rows early
        const uint32_t need = __reduce_max_sync(0xffffffffu, k + pop);
        if (need > ring.base + kRingRows) ring.flush(a, need - kRingRows, k < room ? k : room, rows, lane);
#pragma unroll
        for (int ww = 0; ww < JMAX / 32; ++ww) {
            uint32_t bits = mu[ww];
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1;
                const bool gather = (mg[ww] >> b) & 1u;
                if (k < room)
                    ring.put(a, k, lane, otag | tslot[32 * ww + b] | (gather ? kGather : 0u));
                ++k;
                if (!COUNT && gather) {
                    // the density sum in list order, as the density pass forms it
                    const R4 rj = tile[32 * ww + b];
                    R dx, dy, dz;
                    const R r2 = q.wrap ? sep2<R, true>(rj, q, L, hL, dx, dy, dz) : sep2<R, false>(rj, q, L, hL, dx, dy, dz);
                    const R qq = Real<R>::sqrt_(r2) * ht.invH;
                    R om = (R)1 - qq;
                    om = om > (R)0 ? om : (R)0;
                    const R om2 = om * om;
                    rho += rj.w * ht.cW * om2 * om2 * om2 * ((R)1 + qq * ((R)6 + qq * (R)(35.0 / 3.0)));
                }
            }
        }
        // rows every active lane has passed
        const uint32_t done = __reduce_min_sync(0xffffffffu, G.act ? k : 0xffffffffu);
        if (done > ring.base) ring.flush(a, done, k < room ? k : room, rows, lane);
    }
    ring.flush(a, __reduce_max_sync(0xffffffffu, k), k < room ? k : room, rows, lane);
    if (COUNT && a.census) {
        const uint32_t kept = __reduce_add_sync(0xffffffffu, G.act ? (k < room ? k : room) : 0u);
        if (lane == 0) {
            atomicAdd(&a.census[0], 32ull * tested);
            atomicAdd(&a.census[1], (unsigned long long)kept);
        }
    }
    if (a.nl_bound) {
        if (G.act) a.nl_cnt[i] = k < room ? k : room;
        if (G.act && k > room) atomicExch(a.nl_retry, 1u);  // the host sizes the lists again
    } else if (G.act && k != room) {
        // the two passes drew different sets: keep the lists consistent, report
        a.nl_cnt[i] = k < room ? k : room;
        set_error(a.err, CRK_EOVERFLOW, a.s.id[i]);
    }
    if (!COUNT && G.act) density_out<R>(a, i, ri, rho);
    });
}

// Density alone (no lists) of gas groups whose particles only feed their
// neighbours' corrections in a hierarchical substep: the same visits, tests
// and terms, in the same order, as the fill pass's density sum.
template <typename R, int JMAX>
__global__ void __launch_bounds__(kBlock) density_only_k(PassArgs a)
{
    using R4 = Vec4<R>;
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t w = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    for_each_item(a.n_ggas, a.ggas_dev, a.queue, Q_DONLY, [&](const uint32_t gi) {
    R4 *tile = reinterpret_cast<R4 *>(smem + (size_t)w * hlist_warp_bytes<R, JMAX>());
    uint8_t *tslot = reinterpret_cast<uint8_t *>(reinterpret_cast<float *>(tile + JMAX) + JMAX);
    const Group G = load_group(a.lv, a.ggas, gi, lane);
    const int I = G.I;
    const uint32_t i = G.i;
    const double Ld = a.boxes[a.lv.slot[I]].L;
    const R L = (R)Ld, hL = (R)(0.5 * Ld);
    const R4 *__restrict__ pm = reinterpret_cast<const R4 *>(a.pm);
    const R4 ri = pm[i];
    const HTarget<R> ht = hydro_target<R>(a.s, i);
    float px, py, pz;
    rel_pos(ri, a.lv, I, Ld, px, py, pz);
    const WarpBox wb = warp_box(px, py, pz, G.act);
    const float Hw = warp_max(G.act ? (float)ht.H : 0.f);
    const float Rc = Hw * 1.0001f + 1e-6f * (float)Ld;
    R rho = 0;
    const uint32_t prow = a.hrow[I];
    const RowOrder order(a.hend[I] - prow);
    for (uint32_t t = 0; t < order.n; ++t) {
        const uint32_t p = prow + order.at(t);
        const uint32_t J = a.hcol[p];
        const float4 fr = a.hfr[p];
        if (out_of_range(wb, fr, a.lv.ex[J], a.lv.ey[J], a.lv.ez[J], Rc)) continue;
        const uint32_t sJ = a.lv.start[J], cJ = a.lv.count[J];
        const uint32_t cm = chunks_in_range(a.lv, J, cJ, wb, fr, Rc);
        if (cm == 0u) continue;
        __syncwarp();
        const uint32_t K = stage_cull<R, false>(tile, tslot, nullptr, pm, nullptr, sJ, cJ, cm, wb,
                                                cand_frame<R>(a.lv, I, fr, Ld), Rc, lane);
        __syncwarp();
        if (K == 0u) continue;
        const Target<R> q = target_in_frame(ri, fr);
        uint32_t m[JMAX / 32];
        test_tile_any<R, JMAX, false>(tile, nullptr, q, L, hL, ht.H2, G.act ? chunk_mask(K) : 0u, m);
#pragma unroll
        for (int ww = 0; ww < JMAX / 32; ++ww) {
            uint32_t bits = m[ww];
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1;
                const R4 rj = tile[32 * ww + b];
                R dx, dy, dz;
                const R r2 = q.wrap ? sep2<R, true>(rj, q, L, hL, dx, dy, dz) : sep2<R, false>(rj, q, L, hL, dx, dy, dz);
                const R qq = Real<R>::sqrt_(r2) * ht.invH;
                R om = (R)1 - qq;
                om = om > (R)0 ? om : (R)0;
                const R om2 = om * om;
                rho += rj.w * ht.cW * om2 * om2 * om2 * ((R)1 + qq * ((R)6 + qq * (R)(35.0 / 3.0)));
            }
        }
    }
    if (G.act) density_out<R>(a, i, ri, rho);
    });
}

// Rows of every gas group from the previous step's list sizes (by original
// index): the largest of its targets plus max(16, 1/8) for the particles'
// motion since.  A list that outgrows them makes the fill pass ask for a
// count pass.
__global__ void __launch_bounds__(kBlock) hlist_bound_k(PassArgs a, const uint32_t *__restrict__ cnt_by_id)
{
    const uint32_t lane = threadIdx.x & 31u;
    for_each_item(a.n_ggas, a.ggas_dev, a.queue, Q_HBOUND, [&](const uint32_t gi) {
    const Group G = load_group(a.lv, a.ggas, gi, lane);
    const uint32_t c = __reduce_max_sync(0xffffffffu, G.act ? cnt_by_id[a.s.id[G.i]] : 0u);
    if (lane == 0) a.nl_len[gi] = c + (c / 8u > 16u ? c / 8u : 16u);
    });
}

// Every gas target's list size, stored by original index for the next step.
__global__ void keep_counts_k(PassArgs a, uint32_t *cnt_by_id)
{
    const uint32_t lane = threadIdx.x & 31u;
    for_each_item(a.n_ggas, a.ggas_dev, a.queue, Q_KEEP, [&](const uint32_t gi) {
    const Group G = load_group(a.lv, a.ggas, gi, lane);
    if (G.act) cnt_by_id[a.s.id[G.i]] = a.nl_cnt[G.i];
    });
}

// The neighbour's sorted index and the leaf-pair frame of a list entry.
__device__ __forceinline__ uint32_t entry_index(const uint32_t *hsj_row, uint32_t e)
{
    return hsj_row[(e >> kRowShift) & kMaxRowOffset] + (e & kSlotMask);
}
__device__ __forceinline__ float4 entry_frame(const float4 *frow, uint32_t e)
{
    return frow[(e >> kRowShift) & kMaxRowOffset];
}

// Asks the L2 cache to fetch rows [r0, r1) of a group's list block (row 0
// at g0; rows of 32 entries, 128 bytes, contiguous): one bulk prefetch, no
// completion to wait for.  The rows lie inside the rows the fill wrote.
__device__ __forceinline__ void prefetch_rows(const uint32_t *g0, uint32_t r0, uint32_t r1)
{
    if (r1 <= r0) return;
    const size_t ga = __cvta_generic_to_global(g0 + (size_t)r0 * 32u);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(ga), "r"((r1 - r0) * 128u) : "memory");
}

// Rows of list a consumer asks L2 for ahead of its walk, per prefetch.  The
// lists are written long before they are read and far exceed L2, so every
// row comes from DRAM; a row is fetched 32-64 rows before the walk needs it.
constexpr uint32_t kPrefetchRows = 32;

// Streams a lane's list entries for a consumer that works on entry k while
// the records of entry k + 1 load: entry k + 1's neighbour index was looked
// up one step earlier, entry k + 2's lookup and entry k + 3's load are in
// flight, so that no load is used in the step that issues it.  With PF the
// group's rows themselves are brought to L2 kPrefetchRows at a time, one
// block ahead (density and moments gain; the hydro pass, whose neighbour
// records come from L2, loses by it and does not prefetch).
template <bool PF = true>
struct ListPipe {
    size_t e0;           // the lane's entry 0 (row 0 of its group, column lane)
    uint32_t cnt, rows;  // the lane's entries; the group's longest list
    uint32_t e1, j1;  // the next entry to take and its neighbour index
    uint32_t e2, j2;  // the one after, its index looked up
    uint32_t e3;      // the one after that, loaded

    // on return (e1, j1) is entry 0; every lane of the warp constructs it
    __device__ __forceinline__ ListPipe(const PassArgs &a, uint32_t gi, uint32_t lane, uint32_t n,
                                        const uint32_t *srow)
    {
        const size_t row0 = (size_t)a.nl_row[a.lmap ? a.lmap[gi] : gi];
        e0 = row0 * 32u + lane;
        cnt = n;
        rows = PF ? __reduce_max_sync(0xffffffffu, n) : 0u;
        if (PF && lane == 0) prefetch_rows(a.nl_j + row0 * 32u, 0u, min(rows, 2u * kPrefetchRows));
        e1 = cnt > 0u ? a.nl_j[e0] : 0u;
        e2 = cnt > 1u ? a.nl_j[e0 + 32u] : 0u;
        e3 = cnt > 2u ? a.nl_j[e0 + 64u] : 0u;
        j1 = cnt > 0u ? entry_index(srow, e1) : 0u;
        j2 = cnt > 1u ? entry_index(srow, e2) : 0u;
    }
    // entry m, (e1, j1), was taken: (e1, j1) becomes entry m + 1; with
    // GATHER_ONLY the index of an entry outside the gather set is not looked up
    template <bool GATHER_ONLY = false>
    __device__ __forceinline__ void step(const PassArgs &a, const uint32_t *srow, uint32_t m)
    {
        if (PF && (m % kPrefetchRows) == 0u && m + kPrefetchRows < rows) {
            // the lowest lane still walking asks for the block after next
            const uint32_t act = __activemask(), lane = threadIdx.x & 31u;
            if (lane == (uint32_t)(__ffs(act) - 1))
                prefetch_rows(a.nl_j + (e0 - lane), m + kPrefetchRows, min(rows, m + 2u * kPrefetchRows));
        }
        e1 = e2;
        j1 = j2;
        e2 = e3;
        j2 = (m + 2u < cnt && (!GATHER_ONLY || (e3 & kGather))) ? entry_index(srow, e3) : 0u;
        e3 = m + 3u < cnt ? a.nl_j[e0 + (size_t)(m + 3u) * 32u] : 0u;
    }
};

// Separation x_j - x_i of a listed pair: the neighbour's record moved into
// the target's frame by the leaf-pair frame (FP64: absolute positions).
template <typename R>
__device__ __forceinline__ R list_sep2(const Vec4<R> &rj, const Vec4<R> &ri, const float4 &fr, R L, R hL, R &dx,
                                       R &dy, R &dz)
{
    const Target<R> q = target_in_frame(ri, fr);
    return q.wrap ? sep2<R, true>(rj, q, L, hL, dx, dy, dz) : sep2<R, false>(rj, q, L, hL, dx, dy, dz);
}

// ------------------------------------------------------------- density D

// rho_i = sum_{j in N_i + {i}} m_j W(r, h_i); V = m/rho; P = (gamma-1) rho u^;
// c = sqrt(gamma (gamma-1) u^).  Optional: size and hash of N_i, the FP32
// decision re-taken in FP64 inside the guard band.
template <typename R, int JMAX, bool COUNT>
__global__ void __launch_bounds__(kBlock) density_k(PassArgs a)
{
    using R4 = Vec4<R>;
    const uint32_t lane = threadIdx.x & 31u;
    for_each_item(a.n_ggas, a.ggas_dev, a.queue, Q_DENS, [&](const uint32_t gi) {
    const Group G = load_group(a.lv, a.ggas, gi, lane);
    const int I = G.I;
    const uint32_t i = G.i;
    const R4 *__restrict__ pm = reinterpret_cast<const R4 *>(a.pm);
    const BoxDev &bx = a.boxes[a.lv.slot[I]];
    const double Ld = bx.L;
    const R L = (R)Ld, hL = (R)(0.5 * Ld);
    const R4 ri = pm[i];
    const HTarget<R> ht = hydro_target<R>(a.s, i);
    const float4 *__restrict__ frow = a.hfr + a.hrow[I];
    const uint32_t *__restrict__ srow = a.hsj + a.hrow[I];
    ListPipe<> pipe(a, gi, lane, G.act ? a.nl_cnt[i] : 0u, srow);
    R rho = 0;
    int nc = 0;
    uint64_t hs = 0;
    // the neighbour's record and frame one entry ahead
    R4 rn;
    float4 fn;
    uint32_t en = 0, jn = 0;
    if (pipe.cnt > 0u) {
        en = pipe.e1;
        jn = pipe.j1;
        rn = pm[jn];
        fn = entry_frame(frow, en);
        pipe.step(a, srow, 0u);
    }
    for (uint32_t k = 0; k < pipe.cnt; ++k) {
        const R4 rj = rn;
        const float4 fr = fn;
        const uint32_t e = en;
        const uint32_t j = jn;
        if (k + 1u < pipe.cnt) {
            en = pipe.e1;
            jn = pipe.j1;
            rn = pm[jn];
            fn = entry_frame(frow, en);
            pipe.step(a, srow, k + 1u);
        }
        if (!(e & kGather)) continue;
        R dx, dy, dz;
        const R r2 = list_sep2(rj, ri, fr, L, hL, dx, dy, dz);
        const R r = Real<R>::sqrt_(r2);
        const R qq = r * ht.invH;
        R om = (R)1 - qq;
        om = om > (R)0 ? om : (R)0;
        const R om2 = om * om;
        rho += rj.w * ht.cW * om2 * om2 * om2 * ((R)1 + qq * ((R)6 + qq * (R)(35.0 / 3.0)));
        if (COUNT) {
            bool in = r2 < ht.H2;
            if (Real<R>::mixed) {
                const Target<R> q = target_in_frame(ri, fr);
                const R gb = (R)guard_band((float)ht.H, q.mag);
                if (r2 >= ht.H2 - gb) in = exact_lt(a.s, i, j, Ld, ht.H2x);
            }
            if (in && j != i) {
                ++nc;
                hs += mix64((uint64_t)a.s.id[j]);
            }
        }
    }
    if (!G.act) return;
    density_out<R>(a, i, ri, rho);
    if (COUNT) {
        if (a.nbr_count) a.nbr_count[i] = nc;
        if (a.nbr_hash) a.nbr_hash[i] = hs;
    }
    });
}

// ------------------------------------------------------ correction solve C
// FP64 per particle from the 40 moments (layout: m0, m1[3], m2[xx xy xz yy yz
// zz], dm0[3], dm1[3a+g], dm2[3s+g]):
//   M = m2^-1 (cofactors), singular if |det| < 1e-30 ||m2||_F^3
//   A = 1/(m0 - m1.M m1), B = -M m1,
//   d_g B = -M (d_g m1 + (d_g m2) B)      (= -M d_g m1 - (d_g M) m1)
//   d_g A = -A^2 (d_g m0 + 2 B.d_g m1 + B.(d_g m2) B)
// out: A, B[3], dA[3], dB[9] (dB[3a+g] = d_g B^a).
__device__ bool crk_solve(const double *m, double *out)
{
    const double a00 = m[4], a01 = m[5], a02 = m[6], a11 = m[7], a12 = m[8], a22 = m[9];
    const double c00 = a11 * a22 - a12 * a12;
    const double c01 = a12 * a02 - a01 * a22;
    const double c02 = a01 * a12 - a11 * a02;
    const double c11 = a00 * a22 - a02 * a02;
    const double c12 = a01 * a02 - a00 * a12;
    const double c22 = a00 * a11 - a01 * a01;
    const double det = a00 * c00 + a01 * c01 + a02 * c02;
    const double fro = sqrt(a00 * a00 + a11 * a11 + a22 * a22 + 2.0 * (a01 * a01 + a02 * a02 + a12 * a12));
    if (!(fabs(det) >= 1e-30 * fro * fro * fro) || !(fro > 0.0)) return false;
    const double id = 1.0 / det;
    const double M[3][3] = {{c00 * id, c01 * id, c02 * id},
                            {c01 * id, c11 * id, c12 * id},
                            {c02 * id, c12 * id, c22 * id}};
    const double m1[3] = {m[1], m[2], m[3]};
    double B[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) B[a] = -(M[a][0] * m1[0] + M[a][1] * m1[1] + M[a][2] * m1[2]);
    const double A = 1.0 / (m[0] + B[0] * m1[0] + B[1] * m1[1] + B[2] * m1[2]);
    out[0] = A;
    out[1] = B[0]; out[2] = B[1]; out[3] = B[2];
#pragma unroll
    for (int g = 0; g < 3; ++g) {
        const double dm0 = m[10 + g];
        const double dm1[3] = {m[13 + g], m[16 + g], m[19 + g]};
        const double s0 = m[22 + g], s1 = m[25 + g], s2 = m[28 + g], s3 = m[31 + g], s4 = m[34 + g],
                     s5 = m[37 + g];
        // w = (d_g m2) B
        const double w0 = s0 * B[0] + s1 * B[1] + s2 * B[2];
        const double w1 = s1 * B[0] + s3 * B[1] + s4 * B[2];
        const double w2 = s2 * B[0] + s4 * B[1] + s5 * B[2];
        const double y0 = dm1[0] + w0, y1 = dm1[1] + w1, y2 = dm1[2] + w2;
#pragma unroll
        for (int a = 0; a < 3; ++a) out[7 + 3 * a + g] = -(M[a][0] * y0 + M[a][1] * y1 + M[a][2] * y2);
        const double bdm1 = B[0] * dm1[0] + B[1] * dm1[1] + B[2] * dm1[2];
        const double bw = B[0] * w0 + B[1] * w1 + B[2] * w2;
        out[4 + g] = -A * A * (dm0 + 2.0 * bdm1 + bw);
    }
    return true;
}

// ------------------------------------------------------------- moments M
// Sums over N_i + {i} with W_ij = W(r, h_i), x = x_i - x_j, V_j volumes:
//   m0 += V W, m1^a += V x^a W, m2^ab += V x^a x^b W,
//   d_g m0 += V d_gW, d_g m1^a += V (x^a d_gW + delta_ag W),
//   d_g m2^ab += V (x^a x^b d_gW + (delta_ag x^b + delta_bg x^a) W)
// then the FP64 correction solve; writes hrec2.w = A and hrec3..6.
// The moment sums of one in-range pair, accumulated FMA-first.
template <typename R>
struct MomentAcc {
    R m0, m1[3], m2[6], dm0[3], dm1[9], dm2[18];

    __device__ __forceinline__ void zero()
    {
        m0 = 0;
#pragma unroll
        for (int k = 0; k < 3; ++k) { m1[k] = 0; dm0[k] = 0; }
#pragma unroll
        for (int k = 0; k < 6; ++k) m2[k] = 0;
#pragma unroll
        for (int k = 0; k < 9; ++k) dm1[k] = 0;
#pragma unroll
        for (int k = 0; k < 18; ++k) dm2[k] = 0;
    }

    // x = x_i - x_j, VW = V_j W_ij, Vg = V_j g (V_j grad_i W = Vg x)
    __device__ __forceinline__ void add(const R x[3], R VW, R Vg)
    {
        const R d[3] = {Vg * x[0], Vg * x[1], Vg * x[2]};
        const R xx[6] = {x[0] * x[0], x[0] * x[1], x[0] * x[2], x[1] * x[1], x[1] * x[2], x[2] * x[2]};
        constexpr int SA[6] = {0, 0, 0, 1, 1, 2};  // packed (ab): xx xy xz yy yz zz
        constexpr int SB[6] = {0, 1, 2, 1, 2, 2};
        m0 += VW;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            m1[c] = fma(VW, x[c], m1[c]);
            dm0[c] += d[c];
        }
#pragma unroll
        for (int s = 0; s < 6; ++s) m2[s] = fma(VW, xx[s], m2[s]);
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                dm1[3 * c + q] = fma(x[c], d[q], dm1[3 * c + q]);
                if (c == q) dm1[3 * c + q] += VW;
            }
#pragma unroll
        for (int s = 0; s < 6; ++s)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                R v = fma(xx[s], d[q], dm2[3 * s + q]);
                if (SA[s] == q) v = fma(VW, x[SB[s]], v);
                if (SB[s] == q) v = fma(VW, x[SA[s]], v);
                dm2[3 * s + q] = v;
            }
    }
};

// Mixed form: five CTAs per SM (at most 102 registers a thread).  The few
// registers this spills cost less than the extra warps gain in hiding the
// list and record loads (4.53 -> 3.78 ms at 2x128^3); the FP64 form keeps
// its registers.
template <typename R>
constexpr int moments_min_blocks() { return Real<R>::mixed ? kMomentsMinBlocks : 1; }

template <typename R, int JMAX>
__global__ void __launch_bounds__(kBlock, moments_min_blocks<R>()) moments_k(PassArgs a)
{
    using R4 = Vec4<R>;
    const uint32_t lane = threadIdx.x & 31u;
    for_each_item(a.n_ggas, a.ggas_dev, a.queue, Q_MOM, [&](const uint32_t gi) {
    const Group G = load_group(a.lv, a.ggas, gi, lane);
    const int I = G.I;
    const uint32_t i = G.i;
    const R4 *__restrict__ rec0 = reinterpret_cast<const R4 *>(a.hrec[0]);
    const double Ld = a.boxes[a.lv.slot[I]].L;
    const R L = (R)Ld, hL = (R)(0.5 * Ld);
    const R4 ri = rec0[i];
    const R H = (R)(2.0 * a.s.h[i]);
    const R invH = Real<R>::rcp(H);
    const R invH2 = invH * invH;
    const R cW = (R)kWn * invH2 * invH;
    const R cG = (R)kGn * invH2 * invH2 * invH;
    const float4 *__restrict__ frow = a.hfr + a.hrow[I];
    const uint32_t *__restrict__ srow = a.hsj + a.hrow[I];
    ListPipe<> pipe(a, gi, lane, G.act ? a.nl_cnt[i] : 0u, srow);
    MomentAcc<R> acc;
    acc.zero();
    // the neighbour's record and frame one entry ahead (gather entries only:
    // the moments sum over the gather set, the lists hold the union set)
    R4 rn;
    float4 fn;
    uint32_t en = 0;
    if (pipe.cnt > 0u) {
        en = pipe.e1;
        if (en & kGather) {
            rn = rec0[pipe.j1];
            fn = entry_frame(frow, en);
        }
        pipe.template step<true>(a, srow, 0u);
    }
    for (uint32_t k = 0; k < pipe.cnt; ++k) {
        const R4 rj = rn;
        const float4 fr = fn;
        const uint32_t e = en;
        if (k + 1u < pipe.cnt) {
            en = pipe.e1;
            if (en & kGather) {
                rn = rec0[pipe.j1];
                fn = entry_frame(frow, en);
            }
            pipe.template step<true>(a, srow, k + 1u);
        }
        if (!(e & kGather)) continue;
        R dx, dy, dz;
        const R r2 = list_sep2(rj, ri, fr, L, hL, dx, dy, dz);
        const R x[3] = {-dx, -dy, -dz};
        R Wv, g;
        kernel_wg(Real<R>::sqrt_(r2), invH, cW, cG, Wv, g);
        acc.add(x, rj.w * Wv, rj.w * g);
    }
    if (!G.act) return;
    double m[40];
    m[0] = (double)acc.m0;
#pragma unroll
    for (int c = 0; c < 3; ++c) m[1 + c] = (double)acc.m1[c];
#pragma unroll
    for (int s = 0; s < 6; ++s) m[4 + s] = (double)acc.m2[s];
#pragma unroll
    for (int c = 0; c < 3; ++c) m[10 + c] = (double)acc.dm0[c];
#pragma unroll
    for (int k = 0; k < 9; ++k) m[13 + k] = (double)acc.dm1[k];
#pragma unroll
    for (int k = 0; k < 18; ++k) m[22 + k] = (double)acc.dm2[k];
    double o[16];
    if (!crk_solve(m, o)) {
#pragma unroll
        for (int k = 0; k < 16; ++k) o[k] = 0.0;
        set_error(a.err, CRK_ESINGULAR, a.s.id[i]);
    }
    R4 *rec2 = reinterpret_cast<R4 *>(a.hrec[2]);
    R4 r2v = rec2[i];
    r2v.w = (R)o[0];
    rec2[i] = r2v;
    R4 v3, v4, v5, v6;
    v3.x = (R)o[1]; v3.y = (R)o[2]; v3.z = (R)o[3]; v3.w = (R)o[4];
    v4.x = (R)o[5]; v4.y = (R)o[6]; v4.z = (R)o[7]; v4.w = (R)o[8];
    v5.x = (R)o[9]; v5.y = (R)o[10]; v5.z = (R)o[11]; v5.w = (R)o[12];
    // record 6's free slot carries 1/m_i for the hydro pass's partner side
    v6.x = (R)o[13]; v6.y = (R)o[14]; v6.z = (R)o[15];
    v6.w = Real<R>::rcp(reinterpret_cast<const R4 *>(a.pm)[i].w);
    reinterpret_cast<R4 *>(a.hrec[3])[i] = v3;
    reinterpret_cast<R4 *>(a.hrec[4])[i] = v4;
    reinterpret_cast<R4 *>(a.hrec[5])[i] = v5;
    reinterpret_cast<R4 *>(a.hrec[6])[i] = v6;
    });
}

// Hydro state of one particle, unpacked from its 7 records.
template <typename R>
struct HState {
    R px, py, pz, V;     // position (record frame), volume
    R vx, vy, vz, h;     // predicted velocity, smoothing length
    R rho, P, c, A;
    R B[3], dA[3], dB[9];
};

template <typename R>
__device__ __forceinline__ void unpack_hstate(const Vec4<R> r[7], HState<R> &s)
{
    s.px = r[0].x; s.py = r[0].y; s.pz = r[0].z; s.V = r[0].w;
    s.vx = r[1].x; s.vy = r[1].y; s.vz = r[1].z; s.h = r[1].w;
    s.rho = r[2].x; s.P = r[2].y; s.c = r[2].z; s.A = r[2].w;
    s.B[0] = r[3].x; s.B[1] = r[3].y; s.B[2] = r[3].z; s.dA[0] = r[3].w;
    s.dA[1] = r[4].x; s.dA[2] = r[4].y; s.dB[0] = r[4].z; s.dB[1] = r[4].w;
    s.dB[2] = r[5].x; s.dB[3] = r[5].y; s.dB[4] = r[5].z; s.dB[5] = r[5].w;
    s.dB[6] = r[6].x; s.dB[7] = r[6].y; s.dB[8] = r[6].z;
}

// Corrected kernel gradient of particle s at separation x = x_s - x_other:
//   d_g W^R = A (1 + B.x) g x^g + d_gA (1 + B.x) W + A (sum_a d_gB^a x^a + B^g) W
template <typename R>
__device__ __forceinline__ void corrected_grad(const HState<R> &s, const R x[3], R W, R g, R out[3])
{
    const R lin = (R)1 + s.B[0] * x[0] + s.B[1] * x[1] + s.B[2] * x[2];
    const R Alg = s.A * lin * g;
    const R lW = lin * W;
    const R AW = s.A * W;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const R dBx = s.dB[q] * x[0] + s.dB[3 + q] * x[1] + s.dB[6 + q] * x[2];
        out[q] = Alg * x[q] + s.dA[q] * lW + AW * (dBx + s.B[q]);
    }
}

// --------------------------------------------------------------- hydro H
// Over the hydro pair set (r < H_i or r < H_j, j != i):
//   F_ij = -1/2 V_i V_j (P_i + P_j + Q_i + Q_j) (dW^R_ij - dW^R_ji)
//   Q = rho (-alpha c mu + beta mu^2), mu = min(0, h v_ij.x_ij / (r^2 + eps^2 h^2))
//   m_i a_i = sum F_ij,  m_i du_i = -1/2 sum F_ij . v_ij
// The pairs are the target's list entries; j's seven records are read
// through L1/L2 (a group's neighbours are a few leaves).

// Target side of the hydro pair: the target's state and record 0, and the
// kernel constants of its H = 2h.
template <typename R>
struct HTgt {
    HState<R> s;
    Vec4<R> r0;
    R invH, cW, cG, h2e;
};

template <typename R>
__device__ __forceinline__ void hydro_tgt(HTgt<R> &t, const Vec4<R> r[7], R eps2)
{
    unpack_hstate(r, t.s);
    t.r0 = r[0];
    const R H = (R)2 * t.s.h;
    t.invH = Real<R>::rcp(H);
    t.cW = (R)kWn * t.invH * t.invH * t.invH;
    t.cG = (R)kGn * t.invH * t.invH * t.invH * t.invH * t.invH;
    t.h2e = eps2 * t.s.h * t.s.h;
}

// F_ij and F_ij . v_ij of one listed pair (rn: j's seven records, fr: the
// leaf-pair frame).
template <typename R>
__device__ __forceinline__ void hydro_pair(const HTgt<R> &ti, const Vec4<R> rn[7], const float4 &fr, R L, R hL,
                                           R alpha, R beta, R eps2, R &Fx, R &Fy, R &Fz, R &e)
{
    HState<R> sj;
    unpack_hstate(rn, sj);
    R dx, dy, dz;
    const R r2 = list_sep2(rn[0], ti.r0, fr, L, hL, dx, dy, dz);
    const R x[3] = {-dx, -dy, -dz};  // x_ij = x_i - x_j
    const R xm[3] = {dx, dy, dz};    // x_ji
    const R r = Real<R>::sqrt_(r2);
    R Wi, gi_, Wj, gj;
    kernel_wg(r, ti.invH, ti.cW, ti.cG, Wi, gi_);
    const R invHj = Real<R>::rcp((R)2 * sj.h);
    const R invHj2 = invHj * invHj;
    kernel_wg(r, invHj, (R)kWn * invHj2 * invHj, (R)kGn * invHj2 * invHj2 * invHj, Wj, gj);
    R dWi[3], dWj[3];
    corrected_grad(ti.s, x, Wi, gi_, dWi);
    corrected_grad(sj, xm, Wj, gj, dWj);
    const R vxij = ti.s.vx - sj.vx, vyij = ti.s.vy - sj.vy, vzij = ti.s.vz - sj.vz;
    const R vdx = vxij * x[0] + vyij * x[1] + vzij * x[2];
    R Q = 0;
    if (vdx < (R)0) {
        const R mui = Real<R>::div(ti.s.h * vdx, r2 + ti.h2e);
        const R muj = Real<R>::div(sj.h * vdx, r2 + eps2 * sj.h * sj.h);
        Q = ti.s.rho * (-alpha * ti.s.c * mui + beta * mui * mui) +
            sj.rho * (-alpha * sj.c * muj + beta * muj * muj);
    }
    const R pre = (R)(-0.5) * ti.s.V * sj.V * (ti.s.P + sj.P + Q);
    Fx = pre * (dWi[0] - dWj[0]);
    Fy = pre * (dWi[1] - dWj[1]);
    Fz = pre * (dWi[2] - dWj[2]);
    e = Fx * vxij + Fy * vyij + Fz * vzij;
}

// Walks n list entries of one column of a group's rows, the first at e0,
// one every `stride` words, with the pipeline of ListPipe (entry k + 4's
// word loading, entry k + 3's index being looked up and entry k + 1's
// records loading while entry k is evaluated), and adds the pair sums of
// target ti (sorted index i) to (ax, ay, az, du).
template <typename R>
__device__ __forceinline__ void hydro_walk(const PassArgs &a, const HTgt<R> &ti, uint32_t i, size_t e0,
                                           uint32_t n, uint32_t stride, const float4 *__restrict__ frow,
                                           const uint32_t *__restrict__ srow, R L, R hL, R alpha, R beta, R eps2,
                                           R &ax, R &ay, R &az, R &du)
{
    using R4 = Vec4<R>;
    uint32_t e1 = n > 0u ? a.nl_j[e0] : 0u;
    uint32_t e2 = n > 1u ? a.nl_j[e0 + stride] : 0u;
    uint32_t e3 = n > 2u ? a.nl_j[e0 + 2u * (size_t)stride] : 0u;
    uint32_t j1 = n > 0u ? entry_index(srow, e1) : 0u;
    uint32_t j2 = n > 1u ? entry_index(srow, e2) : 0u;
    // entry m, (e1, j1), was taken: (e1, j1) becomes entry m + 1
    auto step = [&](uint32_t m) {
        e1 = e2;
        j1 = j2;
        e2 = e3;
        j2 = m + 2u < n ? entry_index(srow, e3) : 0u;
        e3 = m + 3u < n ? a.nl_j[e0 + (size_t)(m + 3u) * stride] : 0u;
    };
    // the neighbour's records and frame one entry ahead
    R4 rn[7];
    float4 fn;
    uint32_t jn = 0;
    if (n > 0u) {
        jn = j1;
        fn = entry_frame(frow, e1);
#pragma unroll
        for (int q = 0; q < 7; ++q) rn[q] = reinterpret_cast<const R4 *>(a.hrec[q])[jn];
        step(0u);
    }
    for (uint32_t k = 0; k < n; ++k) {
        const uint32_t j = jn;
        const float4 fr = fn;
        R4 rj[7];
#pragma unroll
        for (int q = 0; q < 7; ++q) rj[q] = rn[q];
        if (k + 1u < n) {
            jn = j1;
            fn = entry_frame(frow, e1);
#pragma unroll
            for (int q = 0; q < 7; ++q) rn[q] = reinterpret_cast<const R4 *>(a.hrec[q])[jn];
            step(k + 1u);
        }
        if (j == i) continue;
        R Fx, Fy, Fz, e;
        hydro_pair(ti, rj, fr, L, hL, alpha, beta, eps2, Fx, Fy, Fz, e);
        ax += Fx;
        ay += Fy;
        az += Fz;
        du += e;
    }
}

// Walk steps a run of the hydro pass's second phase costs beyond its rows
// (the pipeline's restart, the target's records, the tree of shuffles).
constexpr uint32_t kRunSteps = 10;

// Shared memory of a warp of the gather hydro pass: the lanes in order of
// decreasing list length with their lengths, the second phase's sums per
// rank and the first phase's sums per lane (small, so that the carve-out
// leaves L1 to the neighbour records).
template <typename R>
constexpr size_t hydro_warp_bytes()
{
    return 2 * 32 * sizeof(uint32_t) + 2 * 32 * 4 * sizeof(R);
}

// Gather form (each target sums its own pairs, in a fixed order; results do
// not depend on what else runs).  A group's lists differ in length (a
// leaf's last group is often short of targets, and the union sets vary), and
// a warp walking them one lane per target runs as long as its longest list.
// So the walk has two phases: first every lane walks its own list up to
// the length c16 of the 17th longest; then the rows beyond c16 of the 16
// longest lists are spread over the whole warp: while a lists are left (rows
// [c_a, c_{a-1}), c_r the length of the r-th longest), the warp takes q =
// 32 / a rows of them at a time, lane l walking row (l / a) of each q for
// the list of rank l % a, and the q partial sums of a list are added by a
// tree of shuffles.  Each target's sum: its own phase, then the runs in
// order.  A group whose lists are near one length (a uniform box) walks in
// one phase: the two phases are taken only where they save walk steps.
// ONCE (mixed form): each union pair is evaluated by its lower-indexed
// particle only (the union predicate is symmetric, so the pair is in both
// lists): entries with j < i are skipped without loading j's records, the
// target's sums are added once at the end and the partner's side, -F_ij / m_j
// and the same energy term, with one float4 atomic per pair; the outputs
// start from zero.  Results agree with the gather form to rounding.  On
// GB300 the atomics cost more than the halved evaluations save (the lanes of
// a warp skip different entries, so the warp's loop keeps its length; lists
// compacted to the j > i entries first were slower still).
template <typename R, int JMAX, bool ONCE = false>
__global__ void __launch_bounds__(kBlock, Real<R>::mixed ? kHydroMinBlocks : 0) hydro_k(PassArgs a)
{
    using R4 = Vec4<R>;
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t w = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    for_each_item(a.n_ggas, a.ggas_dev, a.queue, Q_HYDRO, [&](const uint32_t gi) {
    const Group G = load_group(a.lv, a.ggas, gi, lane);
    const int I = G.I;
    const uint32_t i = G.i;
    const BoxDev &bx = a.boxes[a.lv.slot[I]];
    const double Ld = bx.L;
    const R L = (R)Ld, hL = (R)(0.5 * Ld);
    const R alpha = (R)bx.av_alpha, beta = (R)bx.av_beta, eps2 = (R)bx.av_eps2;
    const float4 *__restrict__ frow = a.hfr + a.hrow[I];
    const uint32_t *__restrict__ srow = a.hsj + a.hrow[I];
    R4 r[7];
#pragma unroll
    for (int k = 0; k < 7; ++k) r[k] = reinterpret_cast<const R4 *>(a.hrec[k])[i];
    const uint32_t cnt = G.act ? a.nl_cnt[i] : 0u;
    R ax = 0, ay = 0, az = 0, du = 0;
    if constexpr (!ONCE) {
        unsigned char *base = smem + (size_t)w * hydro_warp_bytes<R>();
        uint32_t *sl = reinterpret_cast<uint32_t *>(base);                // lane of rank r
        uint32_t *sc = sl + 32;                                           // length of rank r
        R *acc2 = reinterpret_cast<R *>(sc + 32);                         // [rank][4]
        // rank of the lane's list: longer first, ties by lane
        uint32_t rank = 0;
        for (uint32_t l2 = 0; l2 < 32u; ++l2) {
            const uint32_t c2 = __shfl_sync(0xffffffffu, cnt, (int)l2);
            rank += (c2 > cnt || (c2 == cnt && l2 < lane)) ? 1u : 0u;
        }
        sl[rank] = lane;
        sc[rank] = cnt;
#pragma unroll
        for (int c = 0; c < 4; ++c) acc2[lane * 4 + c] = (R)0;
        __syncwarp();
        // the two phases only where they save steps: the plain walk takes c_0
        // steps, the two phases c16 plus each run's rows / q and a restart
        // of the pipeline (kRunSteps)
        uint32_t c16 = sc[16];
        {
            uint32_t two = c16;
            for (uint32_t na = 16u; na >= 1u; --na) {
                const uint32_t lo = sc[na], hi = sc[na - 1u], q = 32u / na;
                if (hi > lo) two += (hi - lo + q - 1u) / q + kRunSteps;
            }
            if (two >= sc[0]) c16 = sc[0];  // one phase: every lane walks its whole list
        }
        const size_t row0 = (size_t)a.nl_row[a.lmap ? a.lmap[gi] : gi];
        R *own = acc2 + 32 * 4 + lane * 4;  // phase 1's sums of the lane's target
        // segment 0: phase 1, every lane its own list up to c16; segment s > 0:
        // the run of na = 17 - s lists left (rows [c_na, c_{na-1})), the warp
        // on q = 32 / na rows of them at a time
        for (uint32_t seg = 0; seg <= 16u; ++seg) {
            const uint32_t na = 17u - seg;
            const uint32_t lo = seg == 0u ? 0u : (c16 > sc[na] ? c16 : sc[na]), hi = seg == 0u ? c16 : sc[na - 1u];
            if (seg > 0u && hi <= lo) continue;
            const uint32_t q = seg == 0u ? 1u : 32u / na;
            const uint32_t ro = seg == 0u ? 0u : lane / na;
            const bool on = seg == 0u || lane < q * na;
            const uint32_t col = seg == 0u ? lane : sl[on ? lane - ro * na : 0u];
            const uint32_t first = lo + ro;
            uint32_t n = (on && first < hi) ? (hi - first + q - 1u) / q : 0u;
            if (seg == 0u) n = cnt < c16 ? cnt : c16;
            R px = 0, py = 0, pz = 0, pd = 0;
            {
                // the target's records (the lane's own in phase 1, the run's
                // list owner's after it), reread through L1
                const uint32_t it = seg == 0u ? i : G.s0 + col;
                HTgt<R> tj;
                R4 rt[7];
#pragma unroll
                for (int k = 0; k < 7; ++k) rt[k] = reinterpret_cast<const R4 *>(a.hrec[k])[it];
                hydro_tgt(tj, rt, eps2);
                hydro_walk(a, tj, it, (row0 + first) * 32u + col, n, 32u * q, frow, srow, L, hL, alpha, beta, eps2,
                           px, py, pz, pd);
            }
            if (seg == 0u) {
                own[0] = px;
                own[1] = py;
                own[2] = pz;
                own[3] = pd;
                continue;
            }
            // the q partial sums of each list, by a tree over the row slots
            for (uint32_t d = 1u; d < q; d <<= 1) {
                const R vx = __shfl_down_sync(0xffffffffu, px, (int)(d * na));
                const R vy = __shfl_down_sync(0xffffffffu, py, (int)(d * na));
                const R vz = __shfl_down_sync(0xffffffffu, pz, (int)(d * na));
                const R vd = __shfl_down_sync(0xffffffffu, pd, (int)(d * na));
                if (on && (ro & (2u * d - 1u)) == 0u && ro + d < q) {
                    px += vx;
                    py += vy;
                    pz += vz;
                    pd += vd;
                }
            }
            if (lane < na) {
                acc2[lane * 4 + 0] += px;
                acc2[lane * 4 + 1] += py;
                acc2[lane * 4 + 2] += pz;
                acc2[lane * 4 + 3] += pd;
            }
        }
        __syncwarp();
        ax = own[0];
        ay = own[1];
        az = own[2];
        du = own[3];
        if (rank < 16u) {
            ax += acc2[rank * 4 + 0];
            ay += acc2[rank * 4 + 1];
            az += acc2[rank * 4 + 2];
            du += acc2[rank * 4 + 3];
        }
        __syncwarp();
    } else {
        HTgt<R> ti;
        hydro_tgt(ti, r, eps2);
        ListPipe<false> pipe(a, gi, lane, cnt, srow);
        // the neighbour's records and frame one entry ahead
        R4 rn[7];
        float4 fn;
        uint32_t jn = 0;
        if (pipe.cnt > 0u) {
            jn = pipe.j1;
            fn = entry_frame(frow, pipe.e1);
            if (jn > i) {
#pragma unroll
                for (int q = 0; q < 7; ++q) rn[q] = reinterpret_cast<const R4 *>(a.hrec[q])[jn];
            }
            pipe.step(a, srow, 0u);
        }
        for (uint32_t k = 0; k < pipe.cnt; ++k) {
            const uint32_t j = jn;
            const float4 fr = fn;
            R4 rj[7];
#pragma unroll
            for (int q = 0; q < 7; ++q) rj[q] = rn[q];
            if (k + 1u < pipe.cnt) {
                jn = pipe.j1;
                fn = entry_frame(frow, pipe.e1);
                if (jn > i) {
#pragma unroll
                    for (int q = 0; q < 7; ++q) rn[q] = reinterpret_cast<const R4 *>(a.hrec[q])[jn];
                }
                pipe.step(a, srow, k + 1u);
            }
            if (j <= i) continue;
            R Fx, Fy, Fz, e;
            hydro_pair(ti, rj, fr, L, hL, alpha, beta, eps2, Fx, Fy, Fz, e);
            ax += Fx;
            ay += Fy;
            az += Fz;
            du += e;
            // the partner's side: m_j a_j -= F_ij; m_j du_j gets the same -1/2 F_ij . v_ij
            const R imj = rj[6].w;
            atomicAdd(reinterpret_cast<float4 *>(a.acc_h) + j,
                      make_float4((float)(-Fx * imj), (float)(-Fy * imj), (float)(-Fz * imj),
                                  (float)((R)(-0.5) * e * imj)));
        }
    }
    if (!G.act) return;
    const R mi = reinterpret_cast<const R4 *>(a.pm)[i].w;
    const R imi = Real<R>::rcp(mi);
    R4 o;
    o.x = ax * imi;
    o.y = ay * imi;
    o.z = az * imi;
    o.w = (R)(-0.5) * du * imi;
    if (ONCE) atomicAdd(reinterpret_cast<float4 *>(a.acc_h) + i, make_float4((float)o.x, (float)o.y, (float)o.z,
                                                                           (float)o.w));
    else reinterpret_cast<R4 *>(a.acc_h)[i] = o;
    });
}

// ------------------------------------------------------------- gravity G
// a_i = sum_{j != i, r < r_cut} -G m_j x_ij (r^2 + eps^2)^{-3/2} S(r),
// S(r) = erfc(r / 2r_s) + r / (sqrt(pi) r_s) exp(-r^2 / 4r_s^2).
template <typename R>
__device__ __forceinline__ R split_S(R r, R inv2rs)
{
    if (Real<R>::mixed) {
        const float u = (float)r * (float)inv2rs;
        const float tt = Real<float>::rcp(fmaf(kAsP, u, 1.0f));
        const float poly = tt * (kAs1 + tt * (kAs2 + tt * (kAs3 + tt * (kAs4 + tt * kAs5))));
        const float e = Real<float>::exp2(-u * u * kLog2e);  // exp(-u^2) = 2^(-u^2 log2 e)
        return (R)(e * (poly + (float)kTwoOverSqrtPi * u));
    } else {
        const double u = (double)r * (double)inv2rs;
        return (R)(erfc(u) + kTwoOverSqrtPi * u * exp(-u * u));
    }
}

// The pair forces of the K staged candidates of one visit on this lane's
// target, masked by the gravity predicate: r^2 < r_cut^2 in the pass's
// precision, re-decided in FP64 inside the mixed form's guard band.  The
// target itself adds f * (0, 0, 0) = 0 (e2 = max(eps^2, 1e-24) keeps f finite
// when eps = 0 and leaves every other r^2 + eps^2 unchanged in FP32 and FP64);
// only the neighbour count and hash exclude it explicitly.  A lane without a
// target (act false) computes a duplicate of lane 0's sums that is never
// stored.  Staged w: FP64 G m_j; mixed log2(G m_j), so that
// G m_j exp(-u^2) = 2^(log2(G m_j) - v^2) in one ex2.
constexpr float kMinS2 = 1e-24f;

// The plain form's S(r) from the box's series S = 1 - u^3 Q(u^2) (no erfc or
// exp: Q's coefficients, staged in the warp's shared memory, by Horner's
// rule about q_c), or from erfc and exp when the box has no series.
struct SplitSeries {
    const double *coef;  // warp shared memory
    int deg;
    double c, inv4rs2;
};

__device__ __forceinline__ double split_S_series(double r2, const SplitSeries &ss)
{
    const double s = r2 * ss.inv4rs2;  // u^2
    const double t = s - ss.c;
    double q = ss.coef[ss.deg - 1];
    for (int k = ss.deg - 2; k >= 0; --k) q = fma(q, t, ss.coef[k]);
    return fma(-s * sqrt(s), q, 1.0);
}

template <typename R, bool WRAP, bool COUNT>
__device__ __forceinline__ void gravity_tile(const Vec4<R> *tile, const uint8_t *tslot, uint32_t K,
                                             const Target<R> &q, R L, R hL, R rc2, double rc2x, R gb, R e2,
                                             R inv2rs, bool same, bool act, const State &s, uint32_t i,
                                             uint32_t sJ, double Ld, R &ax, R &ay, R &az, int &nc, uint64_t &hs,
                                             const SplitSeries &ss)
{
    const float kv = (float)inv2rs * (float)kSqrtLog2e;
#pragma unroll 4
    for (uint32_t j = 0; j < K; ++j) {
        const Vec4<R> rj = tile[j];
        R dx, dy, dz;
        const R r2 = sep2<R, WRAP>(rj, q, L, hL, dx, dy, dz);
        const R dr = r2 - rc2;
        bool in = dr < (R)0;
        if (Real<R>::mixed && fabs(dr) < gb)
            in = exact_lt(s, i, sJ + tslot[j], Ld, rc2x);  // rare: pairs at the cut
        if (COUNT && same && sJ + tslot[j] == i) in = false;
        R f;
        if (Real<R>::mixed) {
            const float v = Real<float>::sqrt_((float)r2) * kv;
            const float tt = Real<float>::rcp(fmaf(kAsPv, v, 1.0f));
            const float poly = tt * (kAs1 + tt * (kAs2 + tt * (kAs3 + tt * (kAs4 + tt * kAs5))));
            const float sw = Real<float>::exp2(fmaf(-v, v, (float)rj.w)) * fmaf(kTwoOverSqrtPiV, v, poly);
            const float is = Real<float>::rsqrt((float)(r2 + e2));
            f = (R)(sw * is * is * is);  // G m_j S(r) (r^2 + eps^2)^{-3/2}
        } else if (ss.deg > 0) {
            const double S = split_S_series((double)r2, ss);
            const double is = rsqrt((double)(r2 + e2));
            f = (R)(rj.w * S * (is * is * is));  // rj.w = G m_j
        } else {
            const R S = split_S<R>(Real<R>::sqrt_(r2), inv2rs);
            const R s2 = r2 + e2;
            f = rj.w * S * ((R)1 / (s2 * Real<R>::sqrt_(s2)));  // rj.w = G m_j
        }
        f = in ? f : (R)0;  // a_i += f (x_j - x_i)
        ax += f * dx;
        ay += f * dy;
        az += f * dz;
        if (COUNT && in && act) {
            ++nc;
            hs += mix64((uint64_t)s.id[sJ + tslot[j]]);
        }
    }
}

template <typename R, int JMAX, bool COUNT>
__global__ void __launch_bounds__(kBlock) gravity_k(PassArgs a)
{
    using R4 = Vec4<R>;
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t w = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    for_each_item(a.n_gall, a.gall_dev, a.queue, Q_GRAV, [&](const uint32_t gi) {
    R4 *tile = reinterpret_cast<R4 *>(smem + (size_t)w * tile_warp_bytes<R, JMAX>());
    uint8_t *tslot = reinterpret_cast<uint8_t *>(tile + JMAX);
    const Group G = load_group(a.lv, a.gall, gi, lane);
    const int I = G.I;
    const uint32_t i = G.i;
    const R4 *__restrict__ pm = reinterpret_cast<const R4 *>(a.pm);
    const BoxDev &bx = a.boxes[a.lv.slot[I]];
    const double Ld = bx.L;
    const R L = (R)Ld, hL = (R)(0.5 * Ld);
    const R4 ri = pm[i];
    const double rc2x = __dmul_rn(bx.r_cut, bx.r_cut);
    const R rc = (R)bx.r_cut;
    const R rc2 = Real<R>::mixed ? rc * rc : (R)rc2x;
    const R e2 = (R)fmax(bx.eps_soft * bx.eps_soft, (double)kMinS2);
    const R inv2rs = (R)(0.5 / bx.r_split);
    const R Gc = (R)bx.G;
    float px, py, pz;
    rel_pos(ri, a.lv, I, Ld, px, py, pz);
    const WarpBox wb = warp_box(px, py, pz, G.act);
    const float Rc = (float)bx.r_cut * 1.0001f + 1e-6f * (float)Ld;
    // the plain form's split series of this box, in the warp's shared memory
    SplitSeries ss{nullptr, 0, 0.0, 0.0};
    if (!Real<R>::mixed && bx.q_deg > 0) {
        __shared__ double qcoef[kWarps][kSplitTerms];
        __syncwarp();
        for (int k = (int)lane; k < bx.q_deg; k += 32) qcoef[w][k] = bx.q_coef[k];
        __syncwarp();
        ss = SplitSeries{qcoef[w], bx.q_deg, bx.q_c, bx.q_inv4rs2};
    }
    R ax = 0, ay = 0, az = 0;
    int nc = 0;
    uint64_t hs = 0, tested = 0;
    for (uint32_t p = a.grow[I]; p < a.gend[I]; ++p) {
        const uint32_t J = a.gcol[p];
        const float4 fr = a.gfr[p];
        if (out_of_range(wb, fr, a.lv.ex[J], a.lv.ey[J], a.lv.ez[J], Rc)) continue;
        const uint32_t sJ = a.lv.start[J], cJ = a.lv.count[J];
        const uint32_t cm = chunks_in_range(a.lv, J, cJ, wb, fr, Rc);
        if (cm == 0u) continue;
        __syncwarp();
        const uint32_t K = stage_cull<R, false, Real<R>::mixed>(tile, tslot, nullptr, pm, nullptr, sJ, cJ, cm, wb,
                                                                cand_frame<R>(a.lv, I, fr, Ld), Rc, lane, Gc);
        __syncwarp();
        if (K == 0u) continue;
        if (COUNT) tested += K;
        const Target<R> q = target_in_frame(ri, fr);
        const R gb = Real<R>::mixed ? (R)guard_band((float)rc, q.mag) : (R)0;
        const bool same = J == (uint32_t)I;  // the target itself is among the candidates
        // every staged candidate against every target, branch-free: the pair
        // force is formed for all and kept where r < r_cut (a select, so that
        // nothing computed for an out-of-range pair reaches the sums)
        if (q.wrap) gravity_tile<R, true, COUNT>(tile, tslot, K, q, L, hL, rc2, rc2x, gb, e2, inv2rs, same,
                                                 G.act, a.s, i, sJ, Ld, ax, ay, az, nc, hs, ss);
        else gravity_tile<R, false, COUNT>(tile, tslot, K, q, L, hL, rc2, rc2x, gb, e2, inv2rs, same,
                                           G.act, a.s, i, sJ, Ld, ax, ay, az, nc, hs, ss);
    }
    if (COUNT && a.census && lane == 0) {
        atomicAdd(&a.census[2], 32ull * tested);
        atomicAdd(&a.census[3], (unsigned long long)G.cnt * tested);
    }
    if (!G.act) return;
    R4 o;
    o.x = ax; o.y = ay; o.z = az; o.w = 0;
    reinterpret_cast<R4 *>(a.acc_g)[i] = o;
    if (COUNT) {
        if (a.grav_count) a.grav_count[i] = nc;
        if (a.grav_hash) a.grav_hash[i] = hs;
    }
    });
}

// ------------------------------------------- gravity, each pair evaluated once
// The mixed form's short-range gravity with every unordered pair evaluated
// once (paper Sec. IV-B2, Eq. 1-2 and Algorithm 1: warp splitting, partial
// sums exchanged by shuffles, register accumulation, atomics per leaf
// output).  The warp of a target group of leaf I visits only the neighbour
// leaves J >= I of its row; inside leaf I a pair is done by its
// lower-indexed particle.  The staged candidates of a visit are taken in
// chunks of 32 on a diagonal: at step k lane l pairs its target with
// candidate (l + k) mod 32 of the chunk, so the 32 lanes meet 32 different
// candidates; the candidate's partial sum -sum_i G m_i S(r)/(r^2+eps^2)^{3/2}
// x_ij travels with it from lane to lane by three shuffles a step and, after
// 32 steps, is back in lane l = its own slot, which adds it to the
// candidate's acceleration with one float4 atomic (skipped when no pair was
// in range).  The target's own sum stays in registers and is added once at
// the end.  The candidate test, the guard-band re-decision in FP64 and the
// pair force are those of gravity_k; the summation order of the atomics is
// not fixed, so results agree with the gather form to rounding, not bit for
// bit.  Staged w: G m_j.
//
// Candidates of one visit (a leaf J staged alone: the target's own leaf, or
// a pair that needs a per-pair wrap) are indexed by slot in J (tslot, sJ);
// MERGED candidates, staged from consecutive visits into one stream already
// in the target leaf's frame, by particle index (cidx), so that every chunk
// but the group's last holds 32 candidates.
// The 32 steps of one diagonal chunk.  NEAR (a merged chunk whose every
// candidate lies within r_cut of the whole target box, with the guard band
// to spare): every pair is in range, so the test, its FP64 re-decision and
// the select drop out; a lane without a target adds nothing to the
// candidates' partials through Gmi = 0.
template <bool WRAP, bool SAME, bool MERGED, bool NEAR>
__device__ __forceinline__ void gravity_sym_steps(const PassArgs &a, const Vec4<float> *chunk, const uint8_t *cslot,
                                                  const uint32_t *cix, const Target<float> &q, float L, float hL,
                                                  float rc2, float gb, float e2, float kv, float Gmi, bool act,
                                                  uint32_t i, uint32_t sJ, uint32_t lane, float &ax, float &ay,
                                                  float &az, float &bx, float &by, float &bz)
{
    const uint32_t src = (lane + 1u) & 31u;
    const float Gmj = NEAR ? (act ? Gmi : 0.f) : Gmi;
    uint32_t jj = lane;
#pragma unroll 4
    for (int k = 0; k < 32; ++k) {
        const Vec4<float> rj = chunk[jj];
        float dx, dy, dz;
        const float r2 = sep2<float, WRAP>(rj, q, L, hL, dx, dy, dz);
        bool in = true;
        if (!NEAR) {
            const float dr = r2 - rc2;
            in = dr < 0.f;
            if (fabsf(dr) < gb) {
                // rare: a pair at the cut, re-decided in FP64 (arguments read
                // from the kernel's parameters, not held in registers)
                const BoxDev &bxd = a.boxes[a.s.slot[i]];
                in = exact_lt(a.s, i, MERGED ? cix[jj] : sJ + cslot[jj], bxd.L, __dmul_rn(bxd.r_cut, bxd.r_cut));
            }
            if (SAME) in = in && (sJ + cslot[jj] > i);  // one leaf: the lower index does the pair
            in = in && act;
        }
        const float v = Real<float>::sqrt_(r2) * kv;
        const float tt = Real<float>::rcp(fmaf(kAsPv, v, 1.0f));
        const float poly = tt * (kAs1 + tt * (kAs2 + tt * (kAs3 + tt * (kAs4 + tt * kAs5))));
        const float sw = Real<float>::exp2(-v * v) * fmaf(kTwoOverSqrtPiV, v, poly);  // S(r)
        const float is = Real<float>::rsqrt(r2 + e2);
        float f = sw * is * is * is;  // S(r) (r^2 + eps^2)^{-3/2}
        if (!NEAR) f = in ? f : 0.f;
        const float fi = f * rj.w, fj = f * Gmj;
        ax = fmaf(fi, dx, ax);
        ay = fmaf(fi, dy, ay);
        az = fmaf(fi, dz, az);
        bx = fmaf(-fj, dx, bx);
        by = fmaf(-fj, dy, by);
        bz = fmaf(-fj, dz, bz);
        // hand the candidate's partial to the lane that meets it next
        bx = __shfl_sync(0xffffffffu, bx, src);
        by = __shfl_sync(0xffffffffu, by, src);
        bz = __shfl_sync(0xffffffffu, bz, src);
        jj = (jj + 1u) & 31u;
    }
}

template <bool WRAP, bool SAME, bool MERGED>
__device__ __forceinline__ void gravity_sym_tile(const PassArgs &a, const Vec4<float> *tile, const uint8_t *tslot,
                                                 const uint32_t *cidx, const uint8_t *cnear, uint32_t K,
                                                 const Target<float> &q, float L, float hL, float rc2, float gb,
                                                 float e2, float kv, float Gmi, bool act, uint32_t i, uint32_t sJ,
                                                 uint32_t lane, float &ax, float &ay, float &az,
                                                 float4 *__restrict__ acc)
{
    for (uint32_t c0 = 0; c0 < K; c0 += 32u) {
        const Vec4<float> *chunk = tile + c0;
        const uint8_t *cslot = tslot + c0;
        const uint32_t *cix = cidx + c0;
        float bx = 0.f, by = 0.f, bz = 0.f;
        if (MERGED && __all_sync(0xffffffffu, cnear[c0 + lane] != 0))
            gravity_sym_steps<false, false, true, true>(a, chunk, cslot, cix, q, L, hL, rc2, gb, e2, kv, Gmi, act, i,
                                                        sJ, lane, ax, ay, az, bx, by, bz);
        else
            gravity_sym_steps<WRAP, SAME, MERGED, false>(a, chunk, cslot, cix, q, L, hL, rc2, gb, e2, kv, Gmi, act,
                                                         i, sJ, lane, ax, ay, az, bx, by, bz);
        // after 32 shifts the partial of candidate c0 + lane is in lane
        if (c0 + lane < K && (bx != 0.f || by != 0.f || bz != 0.f))
            atomicAdd(acc + (MERGED ? cix[lane] : sJ + cslot[lane]), make_float4(bx, by, bz, 0.f));
    }
}

// Shared memory of a warp of gravity_sym_k: the merged candidate stream
// (up to 31 carried over plus one leaf's JMAX) with its particle indices, and
// the slots of a visit staged alone.
template <int JMAX>
constexpr size_t sym_warp_bytes()
{
    return (JMAX + 32) * (sizeof(float4) + sizeof(uint32_t) + 1) + JMAX;
}
static_assert(sym_warp_bytes<32>() % 16 == 0 && sym_warp_bytes<64>() % 16 == 0 && sym_warp_bytes<128>() % 16 == 0,
              "each warp's tile starts 16-byte aligned");

// Appends to the merged stream at tile[n0, ...) the candidates of leaf J
// that can reach the warp's target box, moved into the target leaf's frame
// (record + pair frame, rounded once), w = G m_j, their particle indices and
// whether the farthest point of the target box lies below near2 from them;
// returns the new length.  Only for pairs that need no per-pair wrap.
__device__ __forceinline__ uint32_t stage_append(float4 *tile, uint32_t *cidx, uint8_t *cnear, uint32_t n0,
                                                 const Vec4<float> *__restrict__ src, uint32_t sJ, uint32_t cJ,
                                                 uint32_t cm, const WarpBox &wb, const float4 &fr, float Rc,
                                                 float near2, uint32_t lane, float Gc)
{
    uint32_t K = n0;
    const uint32_t nch = (cJ + 31u) / 32u;
    for (uint32_t c = 0; c < nch; ++c) {
        if (!((cm >> c) & 1u)) continue;
        const uint32_t k = 32u * c + lane;
        bool keep = false;
        float x = 0.f, y = 0.f, z = 0.f, wv = 0.f;
        if (k < cJ) {
            const Vec4<float> v = src[sJ + k];
            x = v.x + fr.x;
            y = v.y + fr.y;
            z = v.z + fr.z;
            wv = Gc * v.w;
            keep = box_gap2(wb, x, y, z) < Rc * Rc;
        }
        const uint32_t bal = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            const uint32_t pos = K + __popc(bal & ((1u << lane) - 1u));
            tile[pos] = make_float4(x, y, z, wv);
            cidx[pos] = sJ + k;
            const float fx = fabsf(x - wb.cx) + wb.ex, fy = fabsf(y - wb.cy) + wb.ey, fz = fabsf(z - wb.cz) + wb.ez;
            cnear[pos] = (fx * fx + fy * fy + fz * fz) < near2 ? 1u : 0u;
        }
        K += __popc(bal);
    }
    return K;
}

template <int JMAX>
__global__ void __launch_bounds__(kBlock, 7) gravity_sym_k(const __grid_constant__ PassArgs a)
{
    using R4 = Vec4<float>;
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t w = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    for_each_item(a.n_gall, a.gall_dev, a.queue, Q_GSYM, [&](const uint32_t gi) {
    unsigned char *base = smem + (size_t)w * sym_warp_bytes<JMAX>();
    R4 *tile = reinterpret_cast<R4 *>(base);
    uint32_t *cidx = reinterpret_cast<uint32_t *>(tile + JMAX + 32);
    uint8_t *cnear = reinterpret_cast<uint8_t *>(cidx + JMAX + 32);
    uint8_t *tslot = cnear + JMAX + 32;
    const Group G = load_group(a.lv, a.gall, gi, lane);
    const int I = G.I;
    const uint32_t i = G.i;
    const R4 *__restrict__ pm = reinterpret_cast<const R4 *>(a.pm);
    float4 *__restrict__ acc = reinterpret_cast<float4 *>(a.acc_g);
    const BoxDev &bx = a.boxes[a.lv.slot[I]];
    const double Ld = bx.L;
    const float L = (float)Ld, hL = (float)(0.5 * Ld);
    const R4 ri = pm[i];
    const float rc = (float)bx.r_cut;
    const float rc2 = rc * rc;
    const float e2 = (float)fmax(bx.eps_soft * bx.eps_soft, (double)kMinS2);
    const float Gc = (float)bx.G;
    const float kv = (float)(0.5 / bx.r_split) * (float)kSqrtLog2e;
    const float Gmi = Gc * ri.w;
    float px, py, pz;
    rel_pos(ri, a.lv, I, Ld, px, py, pz);
    const WarpBox wb = warp_box(px, py, pz, G.act);
    const float Rc = (float)bx.r_cut * 1.0001f + 1e-6f * (float)Ld;
    float ax = 0.f, ay = 0.f, az = 0.f;
    // the merged stream: the target in its own leaf's frame, the guard band
    // of the largest pair frame staged into it so far
    Target<float> qI;
    qI.qx = ri.x;
    qI.qy = ri.y;
    qI.qz = ri.z;
    qI.wrap = false;
    qI.mag = 0.f;
    float mag = 0.f;
    uint32_t nm = 0;  // candidates waiting in the stream (< 32 between visits)
    // the row is ascending: start at the first J >= I
    uint32_t p = a.grow[I];
    const uint32_t p1 = a.gend[I];
    {
        uint32_t lo = p, hi = p1;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (a.gcol[mid] < (uint32_t)I) lo = mid + 1;
            else hi = mid;
        }
        p = lo;
    }
    while (true) {
        const bool end = p >= p1;
        bool alone = false;
        uint32_t J = 0, sJ = 0, cJ = 0, cm = 0;
        float4 fr = make_float4(0.f, 0.f, 0.f, 0.f);
        if (!end) {
            J = a.gcol[p];
            fr = a.gfr[p];
            ++p;
            if (out_of_range(wb, fr, a.lv.ex[J], a.lv.ey[J], a.lv.ez[J], Rc)) continue;
            sJ = a.lv.start[J];
            cJ = a.lv.count[J];
            cm = chunks_in_range(a.lv, J, cJ, wb, fr, Rc);
            if (cm == 0u) continue;
            alone = J == (uint32_t)I || fr.w < 0.f;
            if (!alone) {
                // into the merged stream
                __syncwarp();
                mag = fmaxf(mag, fr.w);
                // all-in-range: the farthest target below r_cut by the guard
                // band of this leaf's frame (the FP32 distances err by less)
                const float near2 = rc2 - guard_band(rc, mag);
                nm = stage_append(reinterpret_cast<float4 *>(tile), cidx, cnear, nm, pm, sJ, cJ, cm, wb, fr, Rc,
                                  near2, lane, Gc);
                __syncwarp();
                if (nm < 32u) continue;
            }
        }
        // the stream's full chunks; all of it, padded with far sentinels,
        // before a visit staged alone (the target's own leaf, or a pair that
        // needs a per-pair wrap) and at the end of the row
        const bool all = end || alone;
        const uint32_t full = nm & ~31u;
        if (all && nm > full) {
            if (full + lane >= nm) {
                R4 sv;
                sv.x = sv.y = sv.z = Real<float>::far;
                sv.w = 0.f;
                tile[full + lane] = sv;
                cidx[full + lane] = i;
                cnear[full + lane] = 0;
            }
            __syncwarp();
        }
        const uint32_t upto = all ? nm : full;
        if (upto > 0u)
            gravity_sym_tile<false, false, true>(a, tile, tslot, cidx, cnear, upto, qI, L, hL, rc2, guard_band(rc, mag), e2,
                                                 kv, Gmi, G.act, i, 0u, lane, ax, ay, az, acc);
        if (all) {
            nm = 0;
        } else if (nm > full) {
            // the partial chunk moves to the front
            R4 t;
            uint32_t ti = 0;
            uint8_t tn = 0;
            const bool mv = full + lane < nm;
            if (mv) {
                t = tile[full + lane];
                ti = cidx[full + lane];
                tn = cnear[full + lane];
            }
            __syncwarp();
            if (mv) {
                tile[lane] = t;
                cidx[lane] = ti;
                cnear[lane] = tn;
            }
            nm -= full;
        } else {
            nm = 0;
        }
        if (end) break;
        if (!alone) continue;
        __syncwarp();
        const uint32_t K = stage_cull<float, false, false>(tile, tslot, nullptr, pm, nullptr, sJ, cJ, cm, wb,
                                                           cand_frame<float>(a.lv, I, fr, Ld), Rc, lane, Gc);
        __syncwarp();
        if (K == 0u) continue;
        const Target<float> q = target_in_frame(ri, fr);
        const float gb = guard_band(rc, q.mag);
        if (J == (uint32_t)I) {
            if (q.wrap)
                gravity_sym_tile<true, true, false>(a, tile, tslot, cidx, cnear, K, q, L, hL, rc2, gb, e2, kv, Gmi, G.act,
                                                    i, sJ, lane, ax, ay, az, acc);
            else
                gravity_sym_tile<false, true, false>(a, tile, tslot, cidx, cnear, K, q, L, hL, rc2, gb, e2, kv, Gmi, G.act,
                                                     i, sJ, lane, ax, ay, az, acc);
        } else {
            gravity_sym_tile<true, false, false>(a, tile, tslot, cidx, cnear, K, q, L, hL, rc2, gb, e2, kv, Gmi, G.act, i,
                                                 sJ, lane, ax, ay, az, acc);
        }
    }
    if (G.act) atomicAdd(acc + i, make_float4(ax, ay, az, 0.f));
    });
}

// ------------------------------------------------- friends-of-friends groups
// In situ halo finding (paper Sec. IV-B3) on the solver's own leaves and
// gravity leaf-pair lists: particles of the selected species are linked when
// r < b (decided like every neighbour set: FP32 test, FP64 re-decision inside
// the guard band); groups are the connected components.  Concurrent
// union-find over the sorted particles: a union hangs the root of larger
// original index under the root of smaller original index with a
// compare-and-swap on the root's parent, so the final root of a component is
// its particle of smallest original index.  Every retry loop is bounded.
constexpr int kFofRetries = 1 << 22;

__device__ __forceinline__ uint32_t fof_find(uint32_t *par, uint32_t x)
{
    volatile uint32_t *vp = par;
    for (int it = 0; it < kFofRetries; ++it) {
        const uint32_t p = vp[x];
        if (p == x) return x;
        const uint32_t g = vp[p];
        if (g != p) vp[x] = g;  // path halving: only ever points closer to the root
        x = p;
    }
    return 0xffffffffu;
}

// false when a bound ran out (the caller reports CRK_ETIMEOUT)
__device__ __forceinline__ bool fof_union(uint32_t *par, const uint32_t *id, uint32_t a, uint32_t b)
{
    for (int it = 0; it < kFofRetries; ++it) {
        const uint32_t ra = fof_find(par, a), rb = fof_find(par, b);
        if (ra == 0xffffffffu || rb == 0xffffffffu) return false;
        if (ra == rb) return true;
        const bool a_first = id[ra] < id[rb];
        const uint32_t lo = a_first ? ra : rb, hi = a_first ? rb : ra;
        if (atomicCAS(&par[hi], hi, lo) == hi) return true;
    }
    return false;
}

__global__ void fof_init_k(uint32_t *par, int64_t n)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) par[k] = (uint32_t)k;
}

template <typename R, int JMAX>
__global__ void __launch_bounds__(kBlock) fof_link_k(PassArgs a, uint32_t *par, double b, int mask)
{
    using R4 = Vec4<R>;
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t w = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    const uint32_t gi = blockIdx.x * kWarps + w;
    if (gi >= a.n_gall) return;
    R4 *tile = reinterpret_cast<R4 *>(smem + (size_t)w * JMAX * (sizeof(R4) + 1));
    uint8_t *tslot = reinterpret_cast<uint8_t *>(tile + JMAX);
    const Group G = load_group(a.lv, a.gall, gi, lane);
    const int I = G.I;
    if (!((mask >> a.lv.species[I]) & 1)) return;
    const uint32_t i = G.i;
    const R4 *__restrict__ pm = reinterpret_cast<const R4 *>(a.pm);
    const double Ld = a.boxes[a.lv.slot[I]].L;
    const R L = (R)Ld, hL = (R)(0.5 * Ld);
    const R4 ri = pm[i];
    const double b2x = __dmul_rn(b, b);
    const R bb = (R)b;
    const R b2 = Real<R>::mixed ? bb * bb : (R)b2x;
    float px, py, pz;
    rel_pos(ri, a.lv, I, Ld, px, py, pz);
    const WarpBox wb = warp_box(px, py, pz, G.act);
    const float Rc = (float)b * 1.0001f + 1e-6f * (float)Ld;
    bool ok = true;
    for (uint32_t p = a.grow[I]; p < a.gend[I]; ++p) {
        const uint32_t J = a.gcol[p];
        if (!((mask >> a.lv.species[J]) & 1)) continue;
        const float4 fr = a.gfr[p];
        if (out_of_range(wb, fr, a.lv.ex[J], a.lv.ey[J], a.lv.ez[J], Rc)) continue;
        const uint32_t sJ = a.lv.start[J], cJ = a.lv.count[J];
        const uint32_t cm = chunks_in_range(a.lv, J, cJ, wb, fr, Rc);
        if (cm == 0u) continue;
        __syncwarp();
        const uint32_t K = stage_cull<R, false>(tile, tslot, nullptr, pm, nullptr, sJ, cJ, cm, wb,
                                                cand_frame<R>(a.lv, I, fr, Ld), Rc, lane);
        __syncwarp();
        if (K == 0u) continue;
        const Target<R> q = target_in_frame(ri, fr);
        const R gb = Real<R>::mixed ? (R)guard_band((float)b, q.mag) : (R)0;
        uint32_t m[JMAX / 32];
        test_tile_any<R, JMAX, false>(tile, nullptr, q, L, hL, b2 + gb, G.act ? chunk_mask(K) : 0u, m);
#pragma unroll
        for (int ww = 0; ww < JMAX / 32; ++ww) {
            uint32_t bits = m[ww];
            while (bits) {
                const int j = 32 * ww + __ffs(bits) - 1;
                bits &= bits - 1;
                const uint32_t jg = sJ + tslot[j];
                if (jg <= i) continue;  // each pair once, from its lower index
                if (Real<R>::mixed) {
                    R dx, dy, dz;
                    const R r2 = q.wrap ? sep2<R, true>(tile[j], q, L, hL, dx, dy, dz)
                                        : sep2<R, false>(tile[j], q, L, hL, dx, dy, dz);
                    if (r2 >= b2 - gb && !exact_lt(a.s, i, jg, Ld, b2x)) continue;
                }
                ok = fof_union(par, a.s.id, i, jg) && ok;
            }
        }
    }
    if (!ok) set_error(a.err, CRK_ETIMEOUT, a.s.id[i]);
}

// group[id] = original index of the root (smallest of the group), -1 for the
// other species; roots counted.
__global__ void fof_label_k(State s, uint32_t *par, int64_t n, int mask, int64_t *group,
                            unsigned long long *ngroups, int *err)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const uint32_t o = s.id[k];
    if (!((mask >> s.species[k]) & 1)) {
        group[o] = -1;
        return;
    }
    const uint32_t r = fof_find(par, (uint32_t)k);
    if (r == 0xffffffffu) {
        set_error(err, CRK_ETIMEOUT, o);
        group[o] = -1;
        return;
    }
    group[o] = (int64_t)s.id[r];
    if (r == (uint32_t)k) atomicAdd(ngroups, 1ull);
}

template <typename R, int JMAX>
void fof_dispatch(const PassArgs &a, uint32_t *par, double b, int mask, cudaStream_t st)
{
    if (a.n_gall == 0) return;
    const size_t sm = (size_t)kWarps * JMAX * (sizeof(Vec4<R>) + 1);
    fof_link_k<R, JMAX><<<(a.n_gall + kWarps - 1) / kWarps, kBlock, sm, st>>>(a, par, b, mask);
}

inline unsigned nblocks(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

template <typename K>
void launch_warp_kernel(K kernel, uint32_t ngroups, size_t smem, const PassArgs &a, cudaStream_t st)
{
    if (ngroups == 0) return;
    if (smem > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    unsigned grid = nblocks(ngroups, kWarps);
    if (a.queue) {
        // persistent: as many blocks as the SMs hold at once (ngroups is then
        // an upper bound of the items, whose true count is on the device)
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, smem);
        const unsigned resident = (unsigned)(sms > 0 ? sms : 1) * (unsigned)(per_sm > 0 ? per_sm : 1);
        grid = grid < resident ? grid : resident;
    }
    kernel<<<grid, kBlock, smem, st>>>(a);
}

template <typename R, int JMAX>
void hlist_count_dispatch(const PassArgs &a, bool count, cudaStream_t st)
{
    const size_t sm = (size_t)kWarps * hlist_warp_bytes<R, JMAX>();
    if (count) launch_warp_kernel(hlist_count_k<R, JMAX, true>, a.n_ggas, sm, a, st);
    else launch_warp_kernel(hlist_count_k<R, JMAX, false>, a.n_ggas, sm, a, st);
}

template <typename R, int JMAX>
void density_only_dispatch(const PassArgs &a, cudaStream_t st)
{
    launch_warp_kernel(density_only_k<R, JMAX>, a.n_ggas, (size_t)kWarps * hlist_warp_bytes<R, JMAX>(), a, st);
}

template <typename R, int JMAX>
void fill_dispatch(const PassArgs &a, bool count, cudaStream_t st)
{
    const size_t smf = (size_t)kWarps * hfill_warp_bytes<R, JMAX>();
    if (count) launch_warp_kernel(hlist_fill_k<R, JMAX, true>, a.n_ggas, smf, a, st);
    else launch_warp_kernel(hlist_fill_k<R, JMAX, false>, a.n_ggas, smf, a, st);
}

template <typename R, int JMAX>
void density_eval_dispatch(const PassArgs &a, bool count, cudaStream_t st)
{
    if (count) launch_warp_kernel(density_k<R, JMAX, true>, a.n_ggas, 0, a, st);
    else launch_warp_kernel(density_k<R, JMAX, false>, a.n_ggas, 0, a, st);
}

template <typename R, int JMAX>
void gravity_dispatch(const PassArgs &a, bool count, cudaStream_t st)
{
    const size_t sm = (size_t)kWarps * tile_warp_bytes<R, JMAX>();
    if (count) launch_warp_kernel(gravity_k<R, JMAX, true>, a.n_gall, sm, a, st);
    else launch_warp_kernel(gravity_k<R, JMAX, false>, a.n_gall, sm, a, st);
}

template <typename R, int JMAX>
void moments_dispatch(const PassArgs &a, cudaStream_t st)
{
    launch_warp_kernel(moments_k<R, JMAX>, a.n_ggas, 0, a, st);
}

template <typename R, int JMAX>
void hydro_dispatch(const PassArgs &a, cudaStream_t st)
{
    if (Real<R>::mixed && a.hydro_once) {
        // every contribution is added: the rates start from zero
        cudaMemsetAsync(a.acc_h, 0, (size_t)a.n * sizeof(Vec4<R>), st);
        launch_warp_kernel(hydro_k<R, JMAX, true>, a.n_ggas, 0, a, st);
    } else {
        launch_warp_kernel(hydro_k<R, JMAX, false>, a.n_ggas, (size_t)kWarps * hydro_warp_bytes<R>(), a, st);
    }
}

}  // namespace

void launch_fof(const PassArgs &a, int mixed, int cap, uint32_t *par, double b, int mask, int64_t *group,
                unsigned long long *ngroups, cudaStream_t st)
{
    if (a.n <= 0) return;
    fof_init_k<<<nblocks(a.n, 256), 256, 0, st>>>(par, a.n);
    if (mixed) {
        if (cap == 32) fof_dispatch<float, 32>(a, par, b, mask, st);
        else if (cap == 64) fof_dispatch<float, 64>(a, par, b, mask, st);
        else fof_dispatch<float, 128>(a, par, b, mask, st);
    } else {
        if (cap == 32) fof_dispatch<double, 32>(a, par, b, mask, st);
        else if (cap == 64) fof_dispatch<double, 64>(a, par, b, mask, st);
        else fof_dispatch<double, 128>(a, par, b, mask, st);
    }
    fof_label_k<<<nblocks(a.n, 256), 256, 0, st>>>(a.s, par, a.n, mask, group, ngroups, a.err);
    note_launches(3);
}

void launch_records(const PassArgs &a, int mixed, cudaStream_t st)
{
    if (a.n <= 0) return;
    if (mixed) records_k<float><<<nblocks(a.n, 256), 256, 0, st>>>(a);
    else records_k<double><<<nblocks(a.n, 256), 256, 0, st>>>(a);
    note_launches(1);
}

#define CRK_BY_CAP(FN, ...)                                                  \
    do {                                                                     \
        if (mixed) {                                                         \
            if (cap == 32) FN<float, 32>(__VA_ARGS__);                       \
            else if (cap == 64) FN<float, 64>(__VA_ARGS__);                  \
            else FN<float, 128>(__VA_ARGS__);                                \
        } else {                                                             \
            if (cap == 32) FN<double, 32>(__VA_ARGS__);                      \
            else if (cap == 64) FN<double, 64>(__VA_ARGS__);                 \
            else FN<double, 128>(__VA_ARGS__);                               \
        }                                                                    \
    } while (0)

void launch_hlist_count(const PassArgs &a, int mixed, int cap, bool count, cudaStream_t st)
{
    if (a.n_ggas == 0) return;
    CRK_BY_CAP(hlist_count_dispatch, a, count, st);
    note_launches(1);
}

void launch_hlist_fill(const PassArgs &a, int mixed, int cap, bool count, cudaStream_t st)
{
    if (a.n_ggas == 0) return;
    CRK_BY_CAP(fill_dispatch, a, count, st);
    note_launches(1);
}

void launch_density_eval(const PassArgs &a, int mixed, int cap, bool count, cudaStream_t st)
{
    if (a.n_ggas == 0) return;
    CRK_BY_CAP(density_eval_dispatch, a, count, st);
    note_launches(1);
}

void launch_density_only(const PassArgs &a, int mixed, int cap, cudaStream_t st)
{
    if (a.n_ggas == 0) return;
    CRK_BY_CAP(density_only_dispatch, a, st);
    note_launches(1);
}

void launch_hlist_bound(const PassArgs &a, const uint32_t *cnt_by_id, cudaStream_t st)
{
    if (a.n_ggas == 0) return;
    hlist_bound_k<<<nblocks(a.n_ggas, kWarps), kBlock, 0, st>>>(a, cnt_by_id);
    note_launches(1);
}

void launch_keep_counts(const PassArgs &a, uint32_t *cnt_by_id, cudaStream_t st)
{
    if (a.n_ggas == 0) return;
    keep_counts_k<<<nblocks(a.n_ggas, kWarps), kBlock, 0, st>>>(a, cnt_by_id);
    note_launches(1);
}

void launch_moments(const PassArgs &a, int mixed, int cap, cudaStream_t st)
{
    if (a.n_ggas == 0) return;
    CRK_BY_CAP(moments_dispatch, a, st);
    note_launches(1);
}

void launch_hydro(const PassArgs &a, int mixed, int cap, cudaStream_t st)
{
    if (a.n_ggas == 0) return;
    CRK_BY_CAP(hydro_dispatch, a, st);
    note_launches(1);
}

void launch_gravity(const PassArgs &a, int mixed, int cap, bool count, cudaStream_t st)
{
    if (a.n_gall == 0) return;
    if (mixed && !count && a.grav_once) {
        // every contribution is added: the accelerations start from zero
        cudaMemsetAsync(a.acc_g, 0, (size_t)a.n * sizeof(float4), st);
        if (cap == 32)
            launch_warp_kernel(gravity_sym_k<32>, a.n_gall, (size_t)kWarps * sym_warp_bytes<32>(), a, st);
        else if (cap == 64)
            launch_warp_kernel(gravity_sym_k<64>, a.n_gall, (size_t)kWarps * sym_warp_bytes<64>(), a, st);
        else
            launch_warp_kernel(gravity_sym_k<128>, a.n_gall, (size_t)kWarps * sym_warp_bytes<128>(), a, st);
        note_launches(1);
        return;
    }
    CRK_BY_CAP(gravity_dispatch, a, count, st);
    note_launches(1);
}

#undef CRK_BY_CAP

}  // namespace crk
