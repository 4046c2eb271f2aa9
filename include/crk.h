/*
 * crk.h -- C ABI of libcrk, a single-GPU (GB300, sm_103a) implementation of
 * the short-range particle-particle solver of CRK-HACC (arXiv 2510.03557):
 * base leaves of a spatial tree (Sec. IV-B1), leaf-pair interaction lists
 * (Sec. IV-B1), the CRKSPH passes (Sec. IV-A: density, kernel moments, the
 * linear reproducing-kernel corrections A and B with their gradients, the
 * pairwise-antisymmetric momentum and energy rates with artificial
 * viscosity) and the short-range gravity pair force of the long/short-range
 * split (Sec. IV-A), evaluated as the pair sums of Eq. 1-2, plus a fixed-step
 * kick-drift-kick integrator.
 *
 * Conventions shared by every call:
 *   - Return codes: CRK_OK (0) or a negative CRK_E* code; crk_last_error()
 *     then holds a thread-local message.
 *   - Arrays are in the caller's particle order.  Vectors are AoS: particle i
 *     owns pos[3i .. 3i+2].  Tensors: gradA[3i+g] = d A_i / d x^g,
 *     gradB[9i + 3a + g] = d B_i^a / d x^g.
 *   - `mem` selects where every pointer of a call lives: CRK_MEM_HOST or
 *     CRK_MEM_DEVICE (CUDA device memory of the current device).
 *   - Inputs are copied into library-owned device memory; outputs go to
 *     caller-owned buffers.  Handles are opaque and freed by *_destroy only.
 *   - All GPU work of a crk_sim is ordered on the stream given at creation.
 *     Calls on one crk_sim are not thread-safe; the service calls are.
 *   - Species: CRK_DM particles get gravity only (du/dt = 0, A = B = 0);
 *     CRK_GAS particles get hydro and gravity.
 *   - Positions must lie in [0, L) of their box; max(2 h_max, r_cut) < L/2.
 */
#ifndef CRK_H
#define CRK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes */
#define CRK_OK 0
#define CRK_EINVAL (-1)     /* bad argument, size or precondition */
#define CRK_ENOMEM (-2)     /* device or host allocation failed */
#define CRK_ECUDA (-3)      /* a CUDA runtime call failed */
#define CRK_EOVERFLOW (-4)  /* a leaf or pair-list capacity limit was exceeded */
#define CRK_ESINGULAR (-5)  /* the second-moment matrix m2 of a gas particle is not invertible */
#define CRK_EPENDING (-6)   /* crk_poll: the job has not finished yet */
#define CRK_ETIMEOUT (-7)   /* a bounded wait ran out */
#define CRK_ENOTFOUND (-8)  /* crk_poll: unknown or already collected ticket */
#define CRK_ECANCELED (-9)  /* the job was cancelled (crk_service_cancel) */

/* Precision of the pair passes */
#define CRK_FP64 0          /* every operation in FP64 (the plain form) */
#define CRK_MIXED 1         /* FP32 pair arithmetic on leaf-relative coordinates and FP32
                               accumulation; FP64 masters, drift, 3x3 solve, global sums */

#define CRK_WENDLAND_C4 0   /* smoothing kernel, support H = 2h */

#define CRK_MEM_HOST 0
#define CRK_MEM_DEVICE 1

/* crk_params.flags */
#define CRK_FLAG_GRAVITY_PAIRS_ONCE 2  /* mixed form: short-range gravity with each unordered pair
                                          evaluated once (warp splitting, paper Sec. IV-B2 and
                                          Algorithm 1): partial sums passed between lanes by shuffles
                                          and added with atomics, so results agree with the default
                                          gather form to rounding but are not bit-reproducible run to
                                          run.  Without it every target sums its own pairs in a fixed
                                          order (bit-reproducible; a box gives the same bits alone or
                                          batched).  The FP64 form, counted evaluations (neighbour
                                          counts or hashes asked for), hierarchical substeps and the
                                          service always use the gather form. */

#define CRK_FLAG_NO_GRAPH 4            /* run every step host-sized (see crk_step): no CUDA graph */
#define CRK_FLAG_HYDRO_PAIRS_ONCE 8    /* mixed form: the CRKSPH hydro rates with each union pair
                                          evaluated once, by its lower-indexed particle, and the
                                          partner's side added with an atomic (F_ji = -F_ij and
                                          the same energy term); results agree with the default
                                          form to rounding.  Not in the FP64 form, time-step
                                          bin substeps or the service. */

/* Pair decompositions of the mixed form (crk_autotune_ex): bit sets */
#define CRK_GRAVITY_GATHER 0       /* every pass gathers: each target sums its own pairs (32 threads
                                      per visit of a target group to a neighbour leaf, one per target) */
#define CRK_GRAVITY_PAIRS_ONCE 1   /* gravity: each pair once (32 threads per visit, one pair per thread
                                      per step, both sides updated) */
#define CRK_HYDRO_PAIRS_ONCE 2     /* hydro: each union pair once (the lower-indexed side) */

#define CRK_DM 0
#define CRK_GAS 1

/* Physics of one periodic box (paper Sec. IV-A; constants are inputs). */
typedef struct {
    double box;        /* periodic side L */
    double G;          /* gravitational constant (>= 0) */
    double gamma;      /* adiabatic index of the ideal-gas closure P = (gamma-1) rho u */
    double r_cut;      /* short-range gravity cut-off radius */
    double r_split;    /* Gaussian long/short split scale r_s */
    double eps_soft;   /* Plummer softening length */
    double av_alpha;   /* Monaghan viscosity alpha */
    double av_beta;    /* Monaghan viscosity beta */
    double av_eps2;    /* viscosity regulariser epsilon^2 */
    double u_floor;    /* floor on the gas specific thermal energy */
} crk_physics;

/* Simulation-wide settings. */
typedef struct {
    crk_physics phys;  /* physics for crk_load (crk_load_boxes passes its own per box) */
    int kernel;        /* CRK_WENDLAND_C4 */
    int leaf_cap;      /* leaf capacity C: 32, 64 or 128 particles */
    int precision;     /* CRK_FP64 or CRK_MIXED */
    int cm_level;      /* chaining-mesh Morton level b (2^b bins per side); 0 = automatic */
    int flags;         /* CRK_FLAG_* bits (0: none) */
    int rebuild_every; /* sort particles into new leaves every this many steps (0 or 1: every
                          step); in between, leaves keep their particles and their bounding
                          boxes grow with them, and only the boxes, the leaf hierarchy and the
                          pair lists are recomputed (paper Sec. IV-B1: leaves built once per
                          long step, boxes grown in the substeps).  Loading or adding or
                          removing particles always rebuilds. */
    int pm_grid;       /* long-range gravity on an FP64 particle mesh of pm_grid^3 cells (an even
                          number in [4, 1024]; 0: none, the solver computes the short-range part
                          alone).  With a mesh, every acceleration the handle computes or steps
                          with is short-range + long-range, the long-range part the Newtonian
                          force filtered by the Gaussian split (paper Sec. IV-A: FP64 spectral
                          particle-mesh solver for the long-range force).  One box per handle
                          (crk_load, or crk_load_boxes with nbox = 1); not with the service. */
    int graph_margin_pct; /* steps replayed from a CUDA graph (crk_step): the device buffers hold the
                             sizes of the step before the replays plus this many percent (0: 25);
                             a replay batch that outgrows them runs again host-sized, and the margin
                             of the handle's later batches grows by half */
} crk_params;

/* Outputs of crk_forces.  Every pointer is optional (NULL skips it); all
 * live where `mem` says.  Sizes in particles N of the loaded set. */
typedef struct {
    double *acc;          /* 3N: hydro + short-range gravity acceleration (+ the long-range mesh
                             part when pm_grid > 0) */
    double *dudt;         /* N: du/dt (0 for DM) */
    double *rho;          /* N: density (0 for DM) */
    double *A;            /* N: CRK correction A (0 for DM) */
    double *B;            /* 3N: CRK correction B */
    double *gradA;        /* 3N */
    double *gradB;        /* 9N */
    int32_t *nbr_count;   /* N: size of the hydro gather set {gas j != i : r^2 < (2h_i)^2} */
    uint64_t *nbr_hash;   /* N: sum over that set of splitmix64(original index of j), mod 2^64 */
    int32_t *grav_count;  /* N: size of the gravity set {j != i : r^2 < r_cut^2} */
    uint64_t *grav_hash;  /* N: hash of the gravity set as above */
    int mem;              /* CRK_MEM_HOST or CRK_MEM_DEVICE for every pointer above */
    int reserved;
    double momentum_rate[3];  /* written: sum_i m_i a_i (FP64 reduction; ~0 by antisymmetry) */
    double energy_rate;       /* written: sum_i m_i (v_i . a_i^hydro + du_i/dt) (~0) */
} crk_outputs;

/* Per-phase device times of the calls made while timing is on (CUDA events
 * on the sim's stream), accumulated in milliseconds. */
typedef struct {
    double tree_ms;       /* keys, radix sort, permutation, leaves, bounding boxes (S1) */
    double pairs_ms;      /* leaf hierarchy and leaf-pair lists (S2) */
    double density_ms;    /* D (S3) */
    double moments_ms;    /* M + C fused (S4, S5) */
    double hydro_ms;      /* H (S6) */
    double gravity_ms;    /* G (S7) */
    double kdk_ms;        /* kick, drift, predictor, sums (S8) */
    double total_ms;      /* whole calls */
    int64_t calls;        /* force evaluations timed */
    int64_t pairs_hydro;  /* leaf pairs in the last hydro list (ordered) */
    int64_t pairs_grav;   /* leaf pairs in the last gravity list (ordered) */
    int64_t nleaves;      /* leaves in the last tree */
    int64_t launches;     /* CUDA kernels the library launched in the timed calls */
    double pm_ms;         /* long-range mesh gravity (deposit, FFTs, Green's function, gather) */
    /* Pair-work census of the last force evaluation that counted neighbours
     * (crk_forces with nbr_count, nbr_hash, grav_count or grav_hash set; all
     * 0 before one), in lane slots: a warp tests its up to 32 targets against
     * every candidate it stages, so one staged candidate costs 32 slots
     * whatever the group's size.  Against the in-range pairs of the counts
     * these give the evaluated / algorithmic pair ratios. */
    int64_t tests_hydro;        /* hydro candidate tests of the list fill */
    int64_t list_entries;       /* hydro list entries written (union set, self included) */
    int64_t tests_grav;         /* gravity candidate tests (every pair force is formed) */
    int64_t tests_grav_target;  /* of those, the slots of lanes that have a target */
    int64_t list_slots;         /* lane slots of the list rows (32 per row): the moments pass walks
                                   all of them, the hydro pass fewer where its second phase spreads
                                   a group's long lists over the whole warp */
    /* Step counters since the last crk_set_timing (whether timing is on or
     * not): KDK steps run, of those the steps replayed from a CUDA graph,
     * host synchronisations inside host-sized steps and force evaluations
     * (a replayed step has none; a crk_step call that replays graphs
     * synchronises once at its end), and batches of replayed steps that
     * overflowed a capacity and ran again host-sized. */
    int64_t steps;
    int64_t graph_steps;
    int64_t host_syncs;
    int64_t graph_overflows;
} crk_timings;

typedef struct crk_sim crk_sim;

/* Creates a solver handle bound to the current CUDA device.
 * cuda_stream: a cudaStream_t (NULL = the legacy default stream); every GPU
 * operation of the handle is ordered on it.  Errors: CRK_EINVAL for an
 * unsupported leaf_cap / precision / kernel, CRK_ECUDA, CRK_ENOMEM. */
int crk_create(const crk_params *params, void *cuda_stream, crk_sim **out);

/* Loads one periodic box of n particles with the physics of crk_create's
 * params (copied; replaces any previous load).  pos/vel: 3n AoS; mass, u, h:
 * n; species: n bytes, CRK_DM or CRK_GAS.  h is read for gas only.
 * Errors: CRK_EINVAL (n < 0, a position outside [0, L), non-finite input,
 * or max(2 h_max, r_cut) >= L/2), CRK_ENOMEM, CRK_ECUDA. */
int crk_load(crk_sim *sim, int64_t n, const double *pos, const double *vel, const double *mass,
             const double *u, const double *h, const uint8_t *species, int mem);

/* Loads nbox independent periodic boxes back to back (the batched form):
 * box b holds counts[b] consecutive particles of the arrays and has the
 * physics phys[b].  Boxes never interact; one launch per pass covers all.
 * counts and phys are host arrays.  Errors as crk_load. */
int crk_load_boxes(crk_sim *sim, int nbox, const int64_t *counts, const crk_physics *phys,
                   const double *pos, const double *vel, const double *mass, const double *u,
                   const double *h, const uint8_t *species, int mem);

/* One force evaluation at the current state: tree build, leaf-pair lists,
 * density, moments, corrections, hydro and gravity, with the velocities and
 * energies as loaded (or, after crk_step, the KDK predictor values).
 * Writes the requested outputs in the caller's order.  Errors:
 * CRK_ESINGULAR (message names the first particle), CRK_EOVERFLOW,
 * CRK_ECUDA. */
int crk_forces(crk_sim *sim, crk_outputs *out);

/* nsteps fixed-step kick-drift-kick steps of size dt for every box:
 *   v += dt/2 a; u += dt/2 du; x = wrap(x + dt v);
 *   forces at (x, v + dt/2 a_old, u + dt/2 du_old);
 *   v += dt/2 a; u += dt/2 du    (gas u floored at u_floor each time).
 * If no forces exist yet, one force evaluation at the loaded state comes
 * first.  State stays on the device.
 * With nsteps >= 3 (and no mesh, rebuild_every <= 1, timing off, not
 * CRK_FLAG_NO_GRAPH) the first step runs host-sized and the others as
 * replays of a CUDA graph of two steps (paper Sec. IV-A: the data stay on
 * the GPU for the whole step; here no size reaches the host either): every
 * leaf, pair, target-group and list count stays on the device against
 * capacities taken from the first step with a margin, and the pair passes
 * are persistent launches that drain a device work queue of (leaf, target
 * group) items of every box.  The call synchronises once at its end; if a
 * capacity was exceeded, the state of the replays' start is restored and
 * those steps run again host-sized (results are the same either way).
 * Errors as crk_forces. */
int crk_step(crk_sim *sim, double dt, int nsteps);

/* As crk_step with a per-box step size (dt: host array of nbox values). */
int crk_step_boxes(crk_sim *sim, const double *dt, int nsteps);

/* Copies the current state out in the caller's order (any pointer may be
 * NULL).  pos/vel 3N, u N. */
int crk_get_state(crk_sim *sim, double *pos, double *vel, double *u, int mem);

/* Replaces the positions, velocities and energies of the loaded particles
 * (caller's order; any pointer may be NULL to keep that quantity) and keeps
 * masses, species, h and the rates of the last force evaluation, so a
 * following crk_step continues the KDK from the new state.  Positions must
 * lie in [0, L).  Errors: CRK_EINVAL (bad value; the state is then
 * unspecified until the next crk_load), CRK_ECUDA. */
int crk_set_state(crk_sim *sim, const double *pos, const double *vel, const double *u, int mem);

/* FP64 device reductions of the current state over all boxes:
 * momentum = sum m v, energy = sum (1/2 m v^2 + m u); nfloor = floor events
 * since load. */
int crk_get_sums(crk_sim *sim, double momentum[3], double *energy, int64_t *nfloor);

/* Number of particles and boxes loaded. */
int crk_get_size(crk_sim *sim, int64_t *n, int *nbox);

/* Friends-of-friends groups of the loaded particles: the paper's in situ
 * halo finding on the GPU (Sec. IV-B3), here on the solver's own leaves and
 * gravity leaf-pair lists.  Particles of the species set in species_mask
 * (bit 0: CRK_DM, bit 1: CRK_GAS) are linked when r < b, r^2 formed as for
 * the neighbour sets (FP64, (dx*dx + dy*dy) + dz*dz, dx wrapped once); the
 * mixed form tests in FP32 and re-decides in FP64 inside the guard band, so
 * the links are the FP64 links.  Groups are the connected components.
 * group[i] (caller order, n entries, where mem says) = the smallest original
 * index in i's group, -1 for particles of the other species; *ngroups =
 * number of groups, singletons included.  Requires 0 < b <= r_cut of every
 * box.  Sorts the particles into a new tree for the current state (the state
 * itself is unchanged).  Synchronises the stream.  Errors: CRK_EINVAL,
 * CRK_ECUDA, CRK_ETIMEOUT (a bounded retry loop of the union-find ran out). */
int crk_fof(crk_sim *sim, double b, int species_mask, int64_t *group, int64_t *ngroups, int mem);

/* Long-range gravity alone: the mesh acceleration of every particle at the
 * current positions, acc 3N in load order where `mem` says (paper Sec. IV-A;
 * the particle-mesh steps, all FP64: cloud-in-cell deposit of the mass
 * density on the pm_grid^3 mesh of cell d = L / pm_grid with cell centres at
 * (i + 1/2) d; forward FFT; phi(k) = -4 pi G rho(k) exp(-k^2 r_s^2) /
 * (k^2 C(k)^2) with phi(0) = 0 and C(k) = prod_a sinc^2(k_a d / 2); a(k) =
 * -i k phi(k) per axis, zero on that axis's Nyquist plane; inverse FFTs;
 * cloud-in-cell gather).  The deposit adds in no fixed order, so results
 * agree with any other evaluation to rounding, not bit for bit.  The state
 * and the tree are unchanged.  Synchronises the stream.  Errors: CRK_EINVAL
 * (null handle, pm_grid = 0, bad mem flag), CRK_ENOMEM, CRK_ECUDA. */
int crk_pm_accel(crk_sim *sim, double *acc, int mem);

/* Hierarchical (block) time steps: nlong long steps of dt_long, each cut into
 * 2^depth substeps (paper Sec. II and IV-B1: particles grouped into
 * power-of-two timestep bins that follow local conditions; forces evaluated
 * only for the active leaves of a substep; leaves built once per long step
 * and their boxes grown in its substeps).  A particle in bin b (0..depth)
 * takes steps of dt_long / 2^b starting at multiples of its step.  Substep s:
 * opening kick v += dt_b/2 a, u += dt_b/2 du of the particles whose step
 * starts at s; drift of all by dt_long / 2^depth; forces at the substep's end
 * for the particles whose step ends there (every particle's velocity and u
 * predicted to that time: v + tau a, u + tau du, tau = time since its step
 * started - dt_b/2); closing kick of those; and a new bin for each: the
 * shallowest b with dt_long / 2^b <= min(sqrt(2 eta eps_soft / |a|),
 * courant h / c) (the first term only when eps_soft > 0, the second for gas,
 * c = sqrt(gamma (gamma - 1) u)), at most depth, and never a bin whose steps
 * do not start at that time.  Bins at the start of the call come from the
 * stored rates (a force evaluation first when there are none).  The passes
 * of a substep run only over the leaves holding an active particle (hydro,
 * gravity), their hydro neighbour leaves (corrections) and the neighbours of
 * those (density, lists).  active_counts (optional, host, nlong * 2^depth
 * entries) gets the number of active particles of every substep.  Every
 * state update is FP64 with each product and sum rounded on its own.
 * depth = 0 is crk_step.  With a mesh (pm_grid > 0) the long-range force is
 * integrated on the long step (Sec. IV-A: the PM force once per PM step, the
 * short-range physics in the substeps): every long step is wrapped in two half
 * kicks v += dt_long/2 a_mesh, the mesh acceleration at the positions of its
 * start and of its end, while the substeps, their stored rates and the bins
 * see the short-range and hydro forces alone (evaluated afresh at the start of
 * the call; a later crk_step or crk_forces evaluates the full forces again).
 * Errors: CRK_EINVAL (dt_long <= 0, depth outside [0, 20], nlong < 0, eta or
 * courant <= 0), the errors of crk_step. */
int crk_step_bins(crk_sim *sim, double dt_long, int depth, int nlong, double eta, double courant,
                  int64_t *active_counts);

/* Timestep bin of every particle (load order, n bytes where `mem` says) as
 * the last crk_step_bins left it.  Synchronises the stream. */
int crk_get_bins(crk_sim *sim, uint8_t *bins, int mem);

/* Leaf-capacity autotuner.  The paper sizes its base leaves by hand for its
 * hardware (Sec. IV-B1: several hundred particles per leaf on MI250X); here the
 * best capacity depends on the particle distribution.  Runs one force
 * evaluation of the loaded particles at each candidate capacity caps[k]
 * (each 32, 64 or 128), timed with CUDA events on the handle's stream after a
 * warm-up evaluation, keeps the fastest for the handle's later calls and
 * writes it to *best_cap (optional); ms_out (optional, ncaps entries) gets
 * each candidate's time in milliseconds.  The particle state is unchanged;
 * the stored accelerations are those of the chosen capacity.  Synchronises
 * the stream.  Errors: CRK_EINVAL (bad candidate, no particles), the errors
 * of crk_forces. */
int crk_autotune(crk_sim *sim, const int *caps, int ncaps, int *best_cap, double *ms_out);

/* The autotuner over two axes: leaf capacity (caps, as crk_autotune) and
 * the pair decomposition of the mixed form's gravity and hydro passes (forms:
 * bit sets of CRK_GRAVITY_PAIRS_ONCE and CRK_HYDRO_PAIRS_ONCE, 0 = gather
 * everywhere; the FP64 form and the service gather whatever is chosen).
 * Times one force evaluation at every pair of candidates (after a warm-up
 * one), keeps the fastest for the handle's later calls (its leaf capacity
 * and its CRK_FLAG_GRAVITY_PAIRS_ONCE / CRK_FLAG_HYDRO_PAIRS_ONCE bits) and
 * writes it to *best_cap / *best_form (optional); ms_out (optional, ncaps x
 * nforms entries) gets the time of caps[k] with forms[f] at ms_out[k * nforms
 * + f].  Synchronises the stream.  Errors: CRK_EINVAL (bad candidate, no
 * particles), the errors of crk_forces. */
int crk_autotune_ex(crk_sim *sim, const int *caps, int ncaps, const int *forms, int nforms, int *best_cap,
                    int *best_form, double *ms_out);

/* Leaves and leaf-pair lists of the handle's last tree (paper Sec. IV-B1:
 * base leaves of the spatial tree and the leaf-pair interaction lists), for
 * inspection and tests.  The sizes are written always; every array pointer
 * is an optional caller-owned HOST buffer (NULL skips it), so a first call
 * with NULL arrays gets the sizes.  Particles are in the tree's sorted order:
 * leaf L holds sorted positions leaf_start[L] .. leaf_start[L] +
 * leaf_count[L] - 1, all of one box and one species; order[k] is the
 * original (load-order) index of sorted position k.  A leaf's box is
 * leaf_centre +- leaf_half per axis (periodic: a particle lies in it when its
 * minimum-image offset from the centre is within the half extent).  Row L of
 * a list (CSR: the entries row[L] .. row[L+1] - 1 of col) holds the leaves
 * whose boxes lie within reach of leaf L's (hydro: gas leaves within the
 * larger of the two leaves' max 2h; gravity: all leaves within r_cut), L
 * itself included, in ascending order.  Errors: CRK_EINVAL (null handle or
 * sizes, no tree yet: call crk_forces or crk_step first), CRK_ECUDA.
 * Synchronises the stream. */
typedef struct {
    int64_t n;              /* written: particles */
    int64_t nleaf;          /* written: leaves */
    int64_t npair_hydro;    /* written: entries of the hydro list */
    int64_t npair_grav;     /* written: entries of the gravity list */
    int64_t *order;         /* n */
    uint32_t *leaf_start;   /* nleaf */
    uint32_t *leaf_count;   /* nleaf */
    uint8_t *leaf_species;  /* nleaf: CRK_DM or CRK_GAS */
    double *leaf_centre;    /* 3 nleaf (x, y, z per leaf) */
    float *leaf_half;       /* 3 nleaf: half extents, rounded up */
    uint32_t *hydro_row;    /* nleaf + 1 */
    uint32_t *hydro_col;    /* npair_hydro */
    uint32_t *grav_row;     /* nleaf + 1 */
    uint32_t *grav_col;     /* npair_grav */
} crk_tree;
int crk_get_tree(crk_sim *sim, crk_tree *out);

/* Measured fused-multiply-add throughput of the current device, the
 * denominator of the pair passes' roofline fractions: precision CRK_MIXED
 * times FP32 FMA chains, CRK_FP64 FP64 FMA chains (8 independent chains per
 * thread, every SM filled with resident blocks, a warm-up launch, then 3
 * launches timed with CUDA events on cuda_stream, a cudaStream_t or NULL);
 * *tflops = 2 flop per FMA / time, in TFLOP/s.  Synchronises the stream.
 * Errors: CRK_EINVAL (bad precision, null tflops), CRK_ECUDA. */
int crk_fma_peak(int precision, double *tflops, void *cuda_stream);

/* Turns per-phase CUDA-event timing on (1) or off (0) and resets it and the
 * step counters.  With timing on every step runs host-sized (the phase
 * events are read back per step). */
int crk_set_timing(crk_sim *sim, int enable);
int crk_get_timings(crk_sim *sim, crk_timings *out);

/* Frees every resource of the handle (synchronises its stream first). */
int crk_destroy(crk_sim *sim);

/* ------------------------------------------------------------------ */
/* Service: continuous batching of many small-box force-and-KDK jobs.   */
/* Jobs are sorted by particle count into size classes.  Each class has  */
/* its own host thread, CUDA stream and batched device state: it admits  */
/* its submitted jobs (FIFO) while slots and the shared HBM budget allow,*/
/* keeps every admitted job's particles and tree resident, advances all  */
/* its resident jobs one KDK step per batched launch sequence, and       */
/* publishes each job when its steps are done; new jobs join at the next */
/* step boundary.  The classes step side by side on the device, so a     */
/* small job does not wait for the largest boxes.                        */
/* ------------------------------------------------------------------ */
typedef struct {
    size_t hbm_budget_bytes;   /* admission limit on the device memory of all resident jobs */
    int max_slots;             /* at most this many resident jobs per size class */
    int precision;             /* CRK_MIXED or CRK_FP64 */
    int leaf_cap;              /* 32, 64 or 128 */
    int device;                /* CUDA device ordinal */
    int snapshot_every;        /* copy every resident job's state to host memory after every
                                  this many of its steps (0: never); see crk_service_snapshot */
    int size_classes;          /* number of size classes K in [1, 8] (0: 3).  A job of n particles
                                  goes to class k, the first with n < 8192 * 8^(k+1), or to the
                                  last class (K = 3: n < 65,536; n < 524,288; the rest) */
    int lane_priority;         /* CUDA stream priorities of the classes: 0 all equal; 1 larger classes
                                  higher (their blocks go first when SMs free up, which shortens the
                                  latency tail of the large jobs); -1 smaller classes higher */
    int reserved[1];
} crk_service_params;

typedef struct {
    crk_physics phys;          /* the box's physics */
    int64_t n;                 /* particles */
    const double *pos, *vel, *mass, *u, *h;   /* host arrays, copied by crk_submit */
    const uint8_t *species;
    double dt;                 /* KDK step */
    int nsteps;                /* KDK steps to run in total */
    int steps_done;            /* resuming from a snapshot: steps already run, else 0 */
    const double *acc;         /* resuming: accelerations of the snapshot (3n), else NULL */
    const double *dudt;        /* resuming: du/dt of the snapshot (n), else NULL */
} crk_job;

typedef struct {
    double *pos, *vel, *u;     /* caller-owned host buffers (3n, 3n, n) */
    double *acc, *dudt;        /* caller-owned host buffers (3n, n) */
    int64_t n;                 /* written: particles */
    int steps_done;            /* written: KDK steps the snapshot is taken after */
    int reserved;
} crk_job_snapshot;

typedef struct {
    double *pos, *vel, *u;     /* caller-owned host buffers (3n, 3n, n) or NULL */
    int64_t n;                 /* written: particles */
    int64_t latency_ns;        /* written: submit to completion */
    int64_t queue_ns;          /* written: submit to admission */
    int status;                /* written: CRK_OK or the job's error */
    int reserved;
} crk_job_result;

typedef struct crk_service crk_service;

/* Creates the service and starts its host threads (one per size class) on
 * params->device.  Errors: CRK_EINVAL, CRK_ENOMEM, CRK_ECUDA. */
int crk_service_create(const crk_service_params *params, crk_service **out);
/* Copies the job's arrays and enqueues it in its size class; *ticket
 * identifies it.  With snapshot_every > 0 the pinned host buffer of the
 * job's snapshots is allocated here, on the submitting thread (its current
 * device is restored), and the device staging at admission, so the serving
 * loop allocates nothing per step.  Errors: CRK_EINVAL (bad job, or a job
 * that alone exceeds the budget), CRK_ENOMEM.  Thread-safe. */
int crk_submit(crk_service *service, const crk_job *job, uint64_t *ticket);
/* Waits up to timeout_us (0 = do not wait, < 0 = forever) for the job;
 * CRK_EPENDING if still running, CRK_ENOTFOUND for an unknown ticket.  On
 * completion copies the final state and frees the ticket.  Thread-safe. */
int crk_poll(crk_service *service, uint64_t ticket, crk_job_result *result, int64_t timeout_us);
/* Stops the service thread after the resident jobs finish and frees it. */
int crk_service_destroy(crk_service *service);
/* Checkpointing (the analogue of the paper's checkpoint/restart tier,
 * Sec. IV-B4, for resident jobs): with snapshot_every = K > 0 the service
 * copies a job's full dynamic state (positions, velocities, u and the
 * accelerations and du/dt of its last force evaluation, in the job's particle
 * order) to host memory after every K of its steps; the device-to-host copy
 * runs on a side stream beside the next step.  crk_service_snapshot writes the
 * latest complete snapshot of a resident, finished or cancelled job whose
 * ticket has not been collected; CRK_EPENDING if none was taken yet.  A job
 * submitted with that state (steps_done, acc, dudt) skips its initial force
 * evaluation and continues exactly where the snapshot was taken: its result is
 * bit-identical to a run without interruption.  Thread-safe. */
int crk_service_snapshot(crk_service *service, uint64_t ticket, crk_job_snapshot *out);
/* Cancels every queued and resident job at the next step boundary (they end
 * with CRK_ECANCELED; their latest snapshots stay readable until collected).
 * The service keeps running and accepts new jobs.  Thread-safe. */
int crk_service_cancel(crk_service *service);

/* ------------------------------------------------------------------ */
/* Allocation-free neighbour sets.                                      */
/* ------------------------------------------------------------------ */
/* For callers that cannot allocate device memory: code whose GPU memory is
 * owned by another allocator (a framework's caching pool, where a raw
 * cudaMalloc both fragments the pool and synchronises the device) and
 * latency-critical loops where the implicit device synchronisation of
 * cudaMalloc / cudaFree is not acceptable.  The paper has no counterpart;
 * this is a service of the library.
 *
 * Computes, for n particles of one periodic box of side `box`, the size and
 * hash of every gas particle's hydro gather set {gas j != i : r^2 < (2h_i)^2}
 * -- the same definition, exact FP64 predicate and hash as crk_forces'
 * nbr_count / nbr_hash for that box loaded alone (0 for DM particles).
 * pos (3n AoS, in [0, box)), h (n), species (n), count (n) and hash (n) are
 * CUDA device pointers; work is ordered on cuda_stream (a cudaStream_t,
 * NULL = legacy default stream) and the call returns without waiting.
 *
 * It allocates nothing: every temporary lives in one fixed device array of
 * about 6.6 MB inside the library, which every GPU that loads the library
 * holds until the process exits.  The first call on a device looks up that
 * array's device address for the current device; make the first call on each
 * device before any stream capture.  All calls share the one array and it
 * keeps the last call's contents, so calls whose GPU work overlaps (on
 * different streams or threads) race: order them on one stream.
 *
 * Invalid particle values are reported in the outputs, since the call does
 * not wait for the GPU: a particle with a coordinate outside [0, box) (or
 * not finite) gets count -1 and hash 0 and belongs to no other particle's
 * set; a gas particle whose h is not finite, negative, or has 2h >= box/2
 * (where one periodic wrap is no longer the minimum image) gets count -1 and
 * hash 0 while still counting in the sets of the others.
 *
 * Errors (returned; crk_last_error() is not updated by this call):
 * CRK_EINVAL for n < 0, n > CRK_NOALLOC_MAX_N, box <= 0 or a NULL pointer
 * when n > 0; CRK_ECUDA if a launch or the address look-up fails. */
#define CRK_NOALLOC_MAX_N 262144
int crk_neighbours_noalloc(int64_t n, const double *pos, const double *h, const uint8_t *species,
                           double box, int32_t *count, uint64_t *hash, void *cuda_stream);

/* Thread-local message of the last failing call on this thread. */
const char *crk_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CRK_H */
