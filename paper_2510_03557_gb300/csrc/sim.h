// Internal definition of the solver handle shared by the C ABI (crk_api.cpp)
// and the service (service.cpp).  Not part of the public ABI.
#pragma once

#include "crk_internal.h"

#include <algorithm>
#include <string>
#include <vector>

namespace crk {

int fail(int code, const char *fmt, ...);

#define CK(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return ::crk::fail(e_ == cudaErrorMemoryAllocation ? CRK_ENOMEM : CRK_ECUDA, \
                               "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),  \
                               __FILE__, __LINE__);                                     \
    } while (0)

#define RET(call)                    \
    do {                             \
        int r_ = (call);             \
        if (r_ != CRK_OK) return r_; \
    } while (0)

// A device buffer that only grows.
struct DBuf {
    void *p = nullptr;
    size_t bytes = 0;
    int ensure(size_t b);
    int ensure_keep(size_t b, size_t keep, cudaStream_t st);
    int ensure_impl(size_t b);
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    template <typename T> T *as() const { return static_cast<T *>(p); }
};

// Leaf pairs a leaf's hydro and gravity rows hold before the lists are
// walked twice (count, then fill).
constexpr uint32_t kPairCapH = 128, kPairCapG = 256;
// Octree levels of a 21-bit-per-axis Morton key (all of them).
constexpr int kAllLevels = 21;

enum Phase { PH_TREE, PH_PAIRS, PH_D, PH_M, PH_H, PH_G, PH_KDK, PH_KICK, PH_PM, PH_N };

}  // namespace crk

// The opaque handle of include/crk.h.
struct crk_sim {
    using DBuf = crk::DBuf;
    using State = crk::State;
    using Leaves = crk::Leaves;
    using Nodes = crk::Nodes;
    using BoxDev = crk::BoxDev;
    crk_params prm{};
    cudaStream_t st = nullptr;
    int device = 0;
    bool mixed = true;
    int cap = 64;
    int64_t n = 0;
    int nbox = 0;
    int slot_bits = 0;
    std::vector<BoxDev> boxes;
    std::vector<int64_t> box_count;
    bool have_forces = false;
    int64_t n_dead = 0;      // particles of removed pool slots, sorted last and dropped next step
    int64_t cap_n = 0;       // particles the per-particle buffers hold
    bool tree_valid = false; // leaves describe the current particle set (order and membership)
    int since_rebuild = 0;   // steps since the last sort

    // device memory
    DBuf boxes_d;
    DBuf stA[17], stB[17];  // state arrays, double-buffered
    State sa{}, sb{};
    DBuf keys, keys_alt, vals, vals_alt, counts, scan_tmp, flags, flag_scan, scalars;
    DBuf lv_u32[3], lv_sp, lv_c[3], lv_e[3], lv_h, lv_chunk[2];
    DBuf nd_f[7], nd_slot;
    DBuf hrow, grow, hcnt, gcnt, hcol, gcol, hfr, gfr, hsj;
    DBuf pm, hrec[7], uhat, acc_h, acc_g;
    DBuf nbrc, nbrh, gravc, gravh;
    DBuf nl_j, nl_row, nl_len, nl_cnt;  // hydro neighbour lists
    DBuf fof_par;                       // friends-of-friends parents and group count
    DBuf pm_mesh, pm_modes, acc_pm;     // long-range mesh: density + 3 fields, 4 spectra, FP64 3n
    int pm_ng = 0;                      // mesh side of the cuFFT plans (0: none)
    int pm_fwd = 0, pm_inv = 0;         // cuFFT plan handles (real-to-complex, complex-to-real)
    // hierarchical steps: leaf flags (active, moments, density), the four
    // selected group lists (density, moments, hydro, gravity), the list rows of
    // the moments and hydro groups, selection scratch, active counts
    DBuf bflag, bgrp[4], bmap[2], bkeep, bpos, bcount;
    // every gas particle's hydro list size of the last step, by original
    // index: the next step sizes its lists from it instead of a count pass
    DBuf cnt_by_id, nl_retry;
    // pair-work census of the last counted force evaluation (see PassArgs)
    DBuf census;
    uint64_t census_h[4] = {};
    int64_t census_rows = 0;
    DBuf pscr_col, pscr_fr, pscr_st;    // leaf-pair rows of fixed capacity before packing
    int pair_two_pass_left = 0;         // builds left that walk the pair lists twice (after an overflow)
    int bins_bmin = -1;                 // hierarchical substep: smallest active bin (-1: not in a substep)
    bool pm_suspend = false;            // hierarchical steps: forces without the mesh (it kicks on the long step)
    int sort_levels = crk::kAllLevels;  // octree levels below the bins that the next sort orders
    bool cnt_valid = false;
    bool is_pool = false;
    int64_t nl_rows = 0;
    DBuf err, nfloor, partial, sums;
    DBuf staging, in_stage;
    Leaves lv{};
    Nodes nd{};
    int nleaf = 0;
    int64_t npair_h = 0, npair_g = 0;
    DBuf grp_cnt, grp_off, grp_gas, grp_all;  // warp work items of the pair passes
    uint32_t n_ggas = 0, n_gall = 0;
    uint32_t *host_scalars = nullptr;  // pinned: [0] nleaf, [1] hydro pairs, [2] gravity pairs
    int *host_err = nullptr;           // pinned: err[0..1]

    // steps captured as CUDA graphs: a step sized on the device against the
    // capacities of the last host-sized step, two steps per graph (the state
    // buffers swap at every sort), the state snapshot a batch restores after
    // an overflow
    DBuf dz;                            // device sizes block (DevSize words)
    DBuf ds_snap;                       // state snapshot of a batch
    int ds_cap_leaf = 0;
    uint32_t ds_cap_items = 0, ds_cap_rows = 0;
    uint32_t ds_cap_ph = 0, ds_cap_pg = 0;  // entries of the hydro / gravity leaf-pair lists
    bool ds_one_walk = false;           // leaf pairs walked once into fixed rows, then packed
    double ds_margin = 1.25;            // capacity over the last sizes (grows after an overflow)
    cudaStream_t cap_st = nullptr;      // stream the graph is captured on
    cudaGraphExec_t graph = nullptr;
    int64_t graph_launch_nodes = 0;     // kernels of one captured step
    // counters since the last crk_set_timing: host synchronisations inside
    // steps, steps run, steps run as graph replays, overflow recoveries
    int64_t host_syncs = 0, steps_run = 0, graph_steps = 0, graph_overflows = 0;

    // timing
    bool timing = false;
    cudaEvent_t ev[crk::PH_N][2] = {};
    cudaEvent_t ev_all[2] = {};
    double acc_ms[crk::PH_N] = {};
    bool recorded[crk::PH_N] = {};
    double total_ms = 0;
    int64_t calls = 0;
    int64_t launches = 0;
};


namespace crk {

// Pool operations used by the service: a handle whose boxes are slots that
// jobs enter and leave between steps.
int pool_init(crk_sim *s, int max_slots);
int pool_add(crk_sim *s, int slot, const crk_physics &phys, int64_t n, const double *pos,
             const double *vel, const double *mass, const double *u, const double *h,
             const uint8_t *species, const double *acc, const double *dudt);
// Device copy of a slot's state in load order: pos 3n, vel 3n, u n, acc 3n,
// du/dt n (11 n doubles at dev), stream-ordered on the handle's stream.
int pool_snapshot(crk_sim *s, int slot, int64_t n, double *dev);
int pool_extract(crk_sim *s, int slot, int64_t n, double *pos, double *vel, double *u);
int pool_remove(crk_sim *s, int slot, int64_t n);
int pool_step(crk_sim *s, const double *dt_per_slot);

// Long-range mesh gravity (pm.cu): FP64 accelerations of the current state
// into acc (3n doubles, sorted order, or load order when `load_order`), on
// the handle's stream.  Needs prm.pm_grid > 0 and one box.
int pm_accelerations(crk_sim *s, double *acc, bool load_order);
void pm_release(crk_sim *s);
size_t pool_bytes_per_particle(const crk_sim *s);

}  // namespace crk
