// Internal declarations of libcrk (device data layout and kernel launchers).
// Not part of the public ABI; include/crk.h is.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>

#include "../../include/crk.h"

namespace crk {

// 4-vector record of the pass's real type, aligned for one vector load
// (16 B for float, 32 B for double).
template <typename R>
struct alignas(4 * sizeof(R)) Vec4 {
    R x, y, z, w;
};

// Terms of the FP64 short-range factor's polynomial (BoxDev::q_coef).
constexpr int kSplitTerms = 40;

// Per-box physics as the kernels read it (one entry per box slot).
struct BoxDev {
    double L, halfL, G, gamma, r_cut, r_split, eps_soft;
    double av_alpha, av_beta, av_eps2, u_floor;
    double dt, hdt;          // step of the current KDK step (0 for a force-only step)
    int cm_shift;            // sort-key shift that leaves (box, species, chaining-mesh bin)
    int active;              // 0: slot holds no live particles (keys sort them last)
    // the FP64 short-range factor S = 1 - u^3 Q(u^2), u = r / (2 r_s): Q as a
    // polynomial in (u^2 - q_c) of degree q_deg - 1 over the box's range of
    // u^2 (q_deg = 0: S from erfc and exp, for ranges where that form loses
    // too many digits to cancellation)
    int q_deg;
    double q_c, q_inv4rs2;
    double q_coef[kSplitTerms];
};

// Particle state in sorted order, FP64 masters (structure of arrays).
struct State {
    double *x, *y, *z;       // positions in [0, L)
    double *vx, *vy, *vz;    // velocities (after the first half kick: v_half)
    double *u;               // specific thermal energy (gas)
    double *m, *h;           // mass, smoothing length (gas)
    double *ax, *ay, *az;    // acceleration of the last force evaluation
    double *du;              // du/dt of the last force evaluation
    uint8_t *species;        // CRK_DM or CRK_GAS
    uint32_t *slot;          // box index
    uint32_t *id;            // original (load-order) index
    uint8_t *bin;            // timestep bin of the hierarchical steps (steps of D_t / 2^bin)
};

// Leaves: runs of <= leaf_cap consecutive sorted particles of one
// (box, species, chaining-mesh bin).
struct Leaves {
    uint32_t *start, *count, *slot;
    uint8_t *species;
    double *cx, *cy, *cz;    // FP64 bounding-box centres
    float *ex, *ey, *ez;     // half extents, rounded up
    float *hmax;             // max 2h over the leaf's gas particles (0 for DM leaves)
    float4 *clo, *chi;       // boxes of the leaf's 32-particle chunks relative to its centre
                             // (kChunks per leaf, outward-rounded; .w unused)
};

constexpr int kChunks = 4;   // chunks of 32 per leaf (leaf capacity <= 128)

// Implicit binary hierarchy over the leaf array: level l node k covers
// leaves [k << l, min((k+1) << l, nleaf)).
struct Nodes {
    float4 *lo;              // conservative FP32 box: lower corner, w = max H of gas leaves below (0: no gas)
    float4 *hi;              // upper corner, w = box slot as int bits (-1 when the node spans several boxes)
    int levels;
    int64_t level_off[40];   // first node of each level
    int64_t total;
};

// CSR leaf-pair list: row I holds the neighbour leaves J (ascending).
struct PairList {
    uint32_t *row;           // nleaf + 1
    uint32_t *col;
    int64_t capacity;
};

// Device pointers the pair passes read and write (sorted order).  Records
// are 4-vectors of the pass's real type; `pm` = (position, mass) where the
// position is leaf-relative (mixed) or absolute (FP64).
struct PassArgs {
    int64_t n;
    int nleaf;
    const BoxDev *boxes;
    State s;
    Leaves lv;
    // leaf-pair lists: row I of a list holds entries [row[I], end[I]) of its
    // columns (CSR: end = row + 1; rows of fixed capacity: end = row + count)
    const uint32_t *hrow, *hend, *hcol;   // hydro list
    const uint32_t *grow, *gend, *gcol;   // gravity list
    const float4 *hfr, *gfr;       // per-entry leaf-pair frames of the two lists
    const uint32_t *hsj;           // hydro list: first sorted particle of each entry's leaf J
    void *pm;                // R4[n]
    void *hrec[7];           // R4[n] each: hydro records
    void *uhat;              // R[n] predicted u
    void *acc_h;             // R4[n]: hydro acceleration, du/dt
    void *acc_g;             // R4[n]: gravity acceleration
    const double *acc_pm;    // FP64 3n: long-range mesh acceleration (null: no mesh)
    // hierarchical steps: forces at the end of substep bsub (-1: fixed step,
    // the predictor takes the box's dt/2) of 2^bdepth substeps of length bd
    int bsub, bdepth;
    double bd;
    const uint32_t *lmap;    // list row index of every group of ggas (null: the group's own index)
    int32_t *nbr_count;      // optional
    uint64_t *nbr_hash;
    int32_t *grav_count;
    uint64_t *grav_hash;
    // hydro neighbour lists (written by the density pass): entry k of lane l
    // of gas group g at [(nl_row[g] + k) * 32 + l]; an entry is bit 31: r < H_i,
    // bits 7-30: the leaf pair's offset in the target leaf's hydro row,
    // bits 0-6: the neighbour's slot in its leaf
    uint32_t *nl_j;
    uint32_t *nl_row;        // first row of every gas group
    uint32_t *nl_len;        // rows of every gas group (its longest list)
    uint32_t *nl_cnt;        // entries of every particle
    // list rows sized from the previous step's counts (nl_bound 1): the fill
    // pass may use all nl_len[g] rows of its group, writes the true counts
    // and sets *nl_retry when a list does not fit
    int nl_bound;
    uint32_t *nl_retry;
    const uint2 *ggas;       // warp work items (leaf, first offset) of gas leaves
    const uint2 *gall;       // warp work items of all leaves
    uint32_t n_ggas, n_gall;
    // device-side item counts (null: n_ggas / n_gall above) and the work-queue
    // counters of the persistent pass launches (null: one warp per item)
    const uint32_t *ggas_dev, *gall_dev;
    uint32_t *queue;
    int *err;                // [0] code, [1] smallest original index of a failing particle
    unsigned long long *nfloor;  // floor events of the u predictor
    // gravity of the mixed form with each unordered pair evaluated once and
    // the sums added by atomics (1), or the deterministic gather (0)
    int grav_once;
    // hydro rates of the mixed form with each union pair evaluated once and
    // the partner's side added by atomics (1), or the gather (0)
    int hydro_once;
    // pair-work census of a counted evaluation (null otherwise): [0] lane
    // slots of the hydro candidate tests (32 x staged candidates per visit),
    // [1] hydro list entries written, [2] lane slots of the gravity tests,
    // [3] of those the slots of lanes with a target
    unsigned long long *census;
};

// Host-side count of kernel launches (every launcher adds what it launched).
void note_launches(int k);
int64_t launches_so_far();

// ---- scan / sort / tree (tree.cu) ----
// Items per tile of the scan and radix-sort kernels, and the scratch words
// those need for n items (a caller sizing fixed scratch uses these too).
constexpr int64_t kSortTile = 4096;
constexpr size_t radix_count_words_for(int64_t n) { return (size_t)256 * (size_t)((n + kSortTile - 1) / kSortTile); }
constexpr size_t scan_tmp_words_for(int64_t n) { return (size_t)((n + kSortTile - 1) / kSortTile) + 1; }
void scan_exclusive_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *total,
                        uint32_t *tmp, cudaStream_t st);
size_t scan_tmp_words(int64_t n);
void radix_sort_u64(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt,
                    int64_t n, uint32_t *counts, uint32_t *scan_tmp, int first_bit, int end_bit,
                    cudaStream_t st, uint64_t **keys_out, uint32_t **vals_out);
size_t radix_count_words(int64_t n);
void launch_morton_keys(const State &s, const BoxDev *boxes, int64_t n, int slot_bits,
                        uint64_t *keys, uint32_t *idx, cudaStream_t st);
void launch_permute(const State &src, const State &dst, const uint32_t *perm, int64_t n,
                    cudaStream_t st);
void launch_leaf_flags(const uint64_t *keys, int slot_bits, const BoxDev *boxes, int64_t n,
                       int cap, uint32_t *flags, int first_bit, uint32_t *stats, cudaStream_t st);
// nl_dev (optional): the leaf count on the device, nleaf then being the
// capacity of the leaf arrays (the launch size); slots beyond the count are
// left empty (no particles, an inverted box, no rows, no groups).
void launch_leaf_kd_order(const State &unsorted, const Leaves &lv, int nleaf, uint32_t *perm,
                          cudaStream_t st, const uint32_t *nl_dev = nullptr);
void launch_leaf_setup(const uint32_t *flags, const uint32_t *scan, int64_t n, int nleaf,
                       Leaves lv, cudaStream_t st, const uint32_t *nl_dev = nullptr);
void launch_leaf_bounds(const State &s, const BoxDev *boxes, Leaves lv, int nleaf, int mixed,
                        void *pm, Nodes nd, cudaStream_t st, const uint32_t *nl_dev = nullptr);
void launch_build_nodes(Nodes &nd, int nleaf, cudaStream_t st);
void launch_group_count(const Leaves &lv, int nleaf, int gas_only, uint32_t *counts, cudaStream_t st,
                        const uint32_t *nl_dev = nullptr);
void launch_group_fill(const Leaves &lv, int nleaf, int gas_only, const uint32_t *off, uint2 *groups,
                       cudaStream_t st, const uint32_t *nl_dev = nullptr);
// mask (optional): leaves without a 1 get an empty row
void launch_pair_count(const Nodes &nd, const Leaves &lv, const BoxDev *boxes, int nleaf,
                       int hydro, uint32_t *counts, cudaStream_t st, const uint8_t *mask = nullptr,
                       const uint32_t *nl_dev = nullptr);
void launch_pair_scratch(const Nodes &nd, const Leaves &lv, const BoxDev *boxes, int nleaf, int hydro,
                         uint32_t *counts, uint32_t cap, uint32_t *col, float4 *frame, uint32_t *start,
                         uint32_t *overflow, cudaStream_t st, const uint8_t *mask = nullptr,
                         const uint32_t *nl_dev = nullptr);
void launch_pair_compact(int nleaf, uint32_t cap, const uint32_t *counts, const uint32_t *row,
                         const uint32_t *scol, const float4 *sframe, const uint32_t *sstart, uint32_t *col,
                         float4 *frame, uint32_t *start, cudaStream_t st, const uint32_t *nl_dev = nullptr);
void launch_pair_fill(const Nodes &nd, const Leaves &lv, const BoxDev *boxes, int nleaf,
                      int hydro, const uint32_t *row, uint32_t *col, float4 *frame, uint32_t *start,
                      cudaStream_t st, const uint8_t *mask = nullptr, const uint32_t *nl_dev = nullptr);

// ---- passes (passes.cu) ----
void launch_records(const PassArgs &a, int mixed, cudaStream_t st);
void launch_hlist_count(const PassArgs &a, int mixed, int cap, bool count, cudaStream_t st);
void launch_hlist_fill(const PassArgs &a, int mixed, int cap, bool count, cudaStream_t st);
void launch_density_eval(const PassArgs &a, int mixed, int cap, bool count, cudaStream_t st);
void launch_density_only(const PassArgs &a, int mixed, int cap, cudaStream_t st);
void launch_hlist_bound(const PassArgs &a, const uint32_t *cnt_by_id, cudaStream_t st);
void launch_keep_counts(const PassArgs &a, uint32_t *cnt_by_id, cudaStream_t st);
void launch_moments(const PassArgs &a, int mixed, int cap, cudaStream_t st);
void launch_hydro(const PassArgs &a, int mixed, int cap, cudaStream_t st);
void launch_gravity(const PassArgs &a, int mixed, int cap, bool count, cudaStream_t st);
void launch_fof(const PassArgs &a, int mixed, int cap, uint32_t *par, double b, int mask, int64_t *group,
                unsigned long long *ngroups, cudaStream_t st);

// ---- integration and outputs (integrate.cu) ----
void launch_kick_drift(const State &s, const BoxDev *boxes, int64_t n,
                       unsigned long long *nfloor, cudaStream_t st);
void launch_final_kick(const PassArgs &a, int mixed, unsigned long long *nfloor, cudaStream_t st);
void launch_rate_sums(const PassArgs &a, int mixed, double *partial, int nblk, double *out6,
                      cudaStream_t st);
void launch_state_sums(const State &s, int64_t n, double *partial, int nblk, double *out6,
                       cudaStream_t st);
int sums_blocks(int64_t n);
void launch_unpermute_outputs(const PassArgs &a, int mixed, double *acc, double *dudt,
                              double *rho, double *A, double *B, double *gA, double *gB,
                              int32_t *nc, uint64_t *nh, int32_t *gc, uint64_t *gh,
                              cudaStream_t st);
void launch_unpermute_state(const State &s, int64_t n, double *pos, double *vel, double *u,
                            cudaStream_t st);
void launch_validate(const State &s, const BoxDev *boxes, int64_t n, int *err, cudaStream_t st);
void launch_set_state(const State &s, int64_t n, const double *pos, const double *vel,
                      const double *u, cudaStream_t st);
void launch_extract_slot(const State &s, int64_t n, uint32_t slot, int64_t n_job, double *pos,
                         double *vel, double *u, double *acc, double *du, cudaStream_t st);
void launch_set_forces(const State &s, int64_t n, const double *acc, const double *du, cudaStream_t st);
void launch_retire_slot(const State &s, int64_t n, uint32_t from, uint32_t to, cudaStream_t st);
void launch_load_state(const State &s, int64_t n, const double *pos, const double *vel,
                       const double *mass, const double *u, const double *h,
                       const uint8_t *species, const uint32_t *slot_of, cudaStream_t st);

// ---- steps sized on the device (integrate.cu) ----
// Words of the device sizes block of a step whose sizes never reach the host
// (the CUDA-graph step): counts written by scans, the overflow bits, and the
// work-queue counters of the persistent pass launches.
enum DevSize {
    DZ_NLEAF_RAW = 0,   // leaves the sort made
    DZ_NLEAF = 1,       // leaves the step uses (0 after an overflow)
    DZ_GGAS = 2,        // gas target groups (0 after an overflow)
    DZ_GALL = 3,        // all target groups (0 after an overflow)
    DZ_ROWS = 4,        // hydro list rows the groups need
    DZ_OVF = 5,         // overflow bits: 1 leaves, 2 leaf pairs, 4 list rows, 8 a list outgrew its rows
    DZ_STATS = 7,       // 2 words: statistics of the leaf cut (unused here)
    DZ_NPH = 10,        // hydro leaf pairs
    DZ_NPG = 11,        // gravity leaf pairs
    DZ_ROW_OVF = 12,    // set by the one-walk pair fill when a leaf's pairs exceed its fixed row
    DZ_QUEUE = 16,      // kQueueSlots words: work-queue heads
    DZ_WORDS = 48
};
constexpr int kQueueSlots = 16;
// stage 0 after the leaf scan (cap: leaf capacity), 1 and 5 after the hydro
// and gravity pair-count scans (cap: their capacities), 6 after a one-walk
// pair fill into fixed rows (flag: its row-overflow word), 2 after the group
// scans, 3 after the list-row scan (cap: row capacity), 4 after the list fill
// (flag: the fill's retry word).  An overflow zeroes the
// counts the rest of the step launches over, so that it touches nothing
// beyond its buffers; the host then restores the state and steps again with
// larger buffers.
void launch_ds_check(uint32_t *dz, int stage, uint32_t cap, const uint32_t *flag, cudaStream_t st);
// ---- hierarchical time steps (bins.cu) ----
void launch_kick_drift_bins(const State &s, const BoxDev *boxes, int64_t n, int sub, int depth, double d,
                            unsigned long long *nfloor, cudaStream_t st);
void launch_close_bins(const PassArgs &a, int mixed, int sub, int depth, double d, double dt_long, double eta,
                       double courant, int b_sync, unsigned long long *nfloor, unsigned long long *nactive,
                       cudaStream_t st);
void launch_assign_bins(const State &s, const BoxDev *boxes, int64_t n, double dt_long, int depth, double eta,
                        double courant, cudaStream_t st);
void launch_leaf_active(const Leaves &lv, int nleaf, const uint8_t *bin, int bmin, uint8_t *flag, cudaStream_t st);
void launch_leaf_expand(const uint32_t *row, const uint32_t *col, int nleaf, const uint8_t *in, uint8_t *out,
                        cudaStream_t st);
// items whose leaf has leaf_flag set and, when given, exclude not set
void launch_group_select(const uint2 *groups, uint32_t n, const uint8_t *leaf_flag, uint32_t *keep, uint32_t *pos,
                         uint32_t *total, uint32_t *tmp, uint2 *out, uint32_t *map, cudaStream_t st,
                         const uint8_t *exclude = nullptr);
void launch_unpermute_bins(const State &s, int64_t n, uint8_t *out, cudaStream_t st);
void launch_pm_kick(const State &s, const double *acc, int64_t n, double hdt, cudaStream_t st);

}  // namespace crk
