// crk_neighbours_noalloc: the hydro gather-set sizes and hashes of one
// periodic box computed with no memory allocation at all.
//
// Some callers cannot allocate: code whose device memory belongs to another
// allocator (a framework's caching pool, where a raw cudaMalloc both
// fragments the pool and synchronises the device) and latency-critical loops
// in which the implicit device synchronisation of cudaMalloc / cudaFree is
// not acceptable.  This entry point keeps every temporary (cell keys, the
// radix-sort buffers and histograms, the cell-size scalar) in one file-scope
// device array of fixed size, so the caller passes only its inputs and
// outputs.
#include "crk_internal.h"

#include <mutex>

namespace crk {

namespace {

constexpr int64_t kMaxN = CRK_NOALLOC_MAX_N;
constexpr int kT = 256;
constexpr size_t kAlign = 256;

constexpr size_t align_up(size_t b) { return (b + kAlign - 1) / kAlign * kAlign; }

// Layout of the scratch array for kMaxN particles.
constexpr size_t kKeysBytes = align_up(kMaxN * sizeof(uint64_t));
constexpr size_t kValsBytes = align_up(kMaxN * sizeof(uint32_t));
// the radix sort's histogram words for kMaxN keys, and the scan scratch of
// its scans over those words (sized by the sort's own formulas)
constexpr size_t kCountWords = radix_count_words_for(kMaxN);
constexpr size_t kCountBytes = align_up(kCountWords * sizeof(uint32_t));
constexpr size_t kScanWords = scan_tmp_words_for((int64_t)kCountWords) + 8;
constexpr size_t kScanBytes = align_up(kScanWords * sizeof(uint32_t));
static_assert(kCountWords >= radix_count_words_for(kMaxN), "histogram area too small");
static_assert(kScanWords >= scan_tmp_words_for((int64_t)kCountWords), "scan area too small");
constexpr size_t kParamBytes = kAlign;  // [0] max 2h bits (u64), [8] cells per side (int)
constexpr size_t kOffKeys = 0;
constexpr size_t kOffKeysAlt = kOffKeys + kKeysBytes;
constexpr size_t kOffVals = kOffKeysAlt + kKeysBytes;
constexpr size_t kOffValsAlt = kOffVals + kValsBytes;
constexpr size_t kOffCounts = kOffValsAlt + kValsBytes;
constexpr size_t kOffScan = kOffCounts + kCountBytes;
constexpr size_t kOffParam = kOffScan + kScanBytes;
constexpr size_t kScratchBytes = kOffParam + kParamBytes;

// The scratch: about 6.6 MB, held by every GPU that loads the library until
// the process exits.  In host code this name is only a stand-in; kernels get
// its device address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mu;
void *g_scratch_ptr[128] = {};  // per device ordinal, filled on its first call

__device__ __forceinline__ uint64_t mix64(uint64_t x)
{
    // SplitMix64 output function (Steele, Lea & Flood 2014).
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// A particle takes part only when its position lies in [0, box) on every
// axis; a gas particle has a set of its own only when 0 <= 2h < box/2 (the
// minimum image of one wrap is then exact).  Anything else, NaN included,
// fails these comparisons.
__device__ __forceinline__ bool pos_ok(const double *pos, int64_t k, double box)
{
    const double x = pos[3 * k], y = pos[3 * k + 1], z = pos[3 * k + 2];
    return x >= 0.0 && x < box && y >= 0.0 && y < box && z >= 0.0 && z < box;
}

__device__ __forceinline__ bool h_ok(double h, double box) { return h >= 0.0 && 2.0 * h < 0.5 * box; }

__global__ void hmax_k(int64_t n, const double *__restrict__ h, const uint8_t *__restrict__ sp,
                       double box, unsigned long long *hbits)
{
    double m = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        if (sp[k] == CRK_GAS && h_ok(h[k], box)) m = fmax(m, 2.0 * h[k]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    // non-negative doubles order like their bit patterns
    if ((threadIdx.x & 31) == 0) atomicMax(hbits, (unsigned long long)__double_as_longlong(m));
}

// Cells per side: the largest count whose cell side exceeds the largest
// support by a relative margin of 1e-9, so that the rounding of a cell index
// (a few ulps) never puts a pair with r < H two cells apart; fewer than three
// cells per side fall back to one cell.
__global__ void cells_k(double box, unsigned char *param)
{
    const double H = __longlong_as_double((long long)*reinterpret_cast<unsigned long long *>(param));
    const double Hm = H * (1.0 + 1e-9);
    int nc = H > 0.0 ? (int)floor(box / Hm) : 1;
    while (nc > 1 && box / (double)nc < Hm) --nc;
    if (nc < 3) nc = 1;
    if (nc > 1024) nc = 1024;
    *reinterpret_cast<int *>(param + 8) = nc;
}

__device__ __forceinline__ int cell_of(double x, double box, int nc)
{
    int c = (int)(x / box * (double)nc);
    return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

__global__ void cell_keys_k(int64_t n, const double *__restrict__ pos, double box,
                            const unsigned char *param, uint64_t *keys, uint32_t *vals)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int nc = *reinterpret_cast<const int *>(param + 8);
    const int cx = cell_of(pos[3 * k], box, nc), cy = cell_of(pos[3 * k + 1], box, nc),
              cz = cell_of(pos[3 * k + 2], box, nc);
    keys[k] = ((uint64_t)cz * nc + cy) * nc + cx;
    vals[k] = (uint32_t)k;
}

__device__ __forceinline__ int64_t lower_bound(const uint64_t *keys, int64_t n, uint64_t v)
{
    int64_t a = 0, b = n;
    while (a < b) {
        const int64_t m = (a + b) >> 1;
        if (keys[m] < v) a = m + 1;
        else b = m;
    }
    return a;
}

// One thread per particle: the gather set {gas j != i : r^2 < (2h_i)^2} with
// the predicate's exact FP64 expression (one wrap, no contraction).  A
// particle that fails pos_ok, or a gas particle that fails h_ok, gets count
// -1 and hash 0; a particle that fails pos_ok is in no other set.
__global__ void gather_k(int64_t n, const double *__restrict__ pos, const double *__restrict__ h,
                         const uint8_t *__restrict__ sp, double box, const unsigned char *param,
                         const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals,
                         int32_t *count, uint64_t *hash)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t cnt = 0;
    uint64_t hs = 0;
    if (!pos_ok(pos, i, box) || (sp[i] == CRK_GAS && !h_ok(h[i], box))) {
        count[i] = -1;
        hash[i] = 0;
        return;
    }
    if (sp[i] == CRK_GAS) {
        const int nc = *reinterpret_cast<const int *>(param + 8);
        const double hL = 0.5 * box;
        const double H = 2.0 * h[i];
        const double H2 = __dmul_rn(H, H);
        const double xi = pos[3 * i], yi = pos[3 * i + 1], zi = pos[3 * i + 2];
        const int cx = cell_of(xi, box, nc), cy = cell_of(yi, box, nc), cz = cell_of(zi, box, nc);
        const int span = nc >= 3 ? 1 : 0;
        for (int dz = -span; dz <= span; ++dz)
            for (int dy = -span; dy <= span; ++dy)
                for (int dx = -span; dx <= span; ++dx) {
                    const int x = (cx + dx + nc) % nc, y = (cy + dy + nc) % nc, z = (cz + dz + nc) % nc;
                    const uint64_t key = ((uint64_t)z * nc + y) * nc + x;
                    for (int64_t k = lower_bound(keys, n, key); k < n && keys[k] == key; ++k) {
                        const uint32_t j = vals[k];
                        if ((int64_t)j == i || sp[j] != CRK_GAS || !pos_ok(pos, j, box)) continue;
                        double ex = pos[3 * (int64_t)j] - xi, ey = pos[3 * (int64_t)j + 1] - yi,
                               ez = pos[3 * (int64_t)j + 2] - zi;
                        if (ex >= hL) ex -= box; else if (ex < -hL) ex += box;
                        if (ey >= hL) ey -= box; else if (ey < -hL) ey += box;
                        if (ez >= hL) ez -= box; else if (ez < -hL) ez += box;
                        const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)),
                                                    __dmul_rn(ez, ez));
                        if (r2 < H2) {
                            ++cnt;
                            hs += mix64((uint64_t)j);
                        }
                    }
                }
    }
    count[i] = cnt;
    hash[i] = hs;
}

// Device address of the scratch on the current device; looked up (without
// allocating) on the first call per device.
int scratch_on_current_device(unsigned char **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) {
        cudaGetLastError();
        return CRK_ECUDA;
    }
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return CRK_ECUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_scratch_ptr[dev]);
    return CRK_OK;
}

}  // namespace

}  // namespace crk

extern "C" int crk_neighbours_noalloc(int64_t n, const double *pos, const double *h,
                                      const uint8_t *species, double box, int32_t *count,
                                      uint64_t *hash, void *cuda_stream)
{
    using namespace crk;
    if (n < 0 || n > kMaxN) return CRK_EINVAL;
    if (!(box > 0.0)) return CRK_EINVAL;
    if (n == 0) return CRK_OK;
    if (!pos || !h || !species || !count || !hash) return CRK_EINVAL;
    unsigned char *base = nullptr;
    const int rc = scratch_on_current_device(&base);
    if (rc != CRK_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    uint64_t *keys = reinterpret_cast<uint64_t *>(base + kOffKeys);
    uint64_t *keys_alt = reinterpret_cast<uint64_t *>(base + kOffKeysAlt);
    uint32_t *vals = reinterpret_cast<uint32_t *>(base + kOffVals);
    uint32_t *vals_alt = reinterpret_cast<uint32_t *>(base + kOffValsAlt);
    uint32_t *counts = reinterpret_cast<uint32_t *>(base + kOffCounts);
    uint32_t *scan = reinterpret_cast<uint32_t *>(base + kOffScan);
    unsigned char *param = base + kOffParam;
    // the running maximum must start at zero on every call
    if (cudaMemsetAsync(param, 0, kParamBytes, st) != cudaSuccess) {
        cudaGetLastError();
        return CRK_ECUDA;
    }
    const unsigned nb = (unsigned)((n + kT - 1) / kT);
    hmax_k<<<nb < 304u ? nb : 304u, kT, 0, st>>>(n, h, species, box,
                                                 reinterpret_cast<unsigned long long *>(param));
    cells_k<<<1, 1, 0, st>>>(box, param);
    cell_keys_k<<<nb, kT, 0, st>>>(n, pos, box, param, keys, vals);
    uint64_t *ko;
    uint32_t *vo;
    // cell ids are below 2^30: four 8-bit passes, ending back in keys / vals
    radix_sort_u64(keys, vals, keys_alt, vals_alt, n, counts, scan, 0, 32, st, &ko, &vo);
    gather_k<<<nb, kT, 0, st>>>(n, pos, h, species, box, param, ko, vo, count, hash);
    note_launches(4);  // hmax, cells, keys, gather (the sort counts its own launches)
    if (cudaGetLastError() != cudaSuccess) return CRK_ECUDA;
    return CRK_OK;
}
