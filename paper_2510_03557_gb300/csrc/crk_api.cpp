// Host side of the C ABI declared in include/crk.h: handle lifetime, input
// checks, device memory, and the per-step launch sequence
//   [kick + drift] -> Morton keys -> radix sort -> permute -> leaves ->
//   leaf hierarchy -> leaf-pair lists -> predictor records -> D -> M+C -> H
//   -> G -> [second kick] -> sums
// all ordered on the handle's stream (paper Sec. IV-A/IV-B: the data stays on
// the device for the whole run; only leaf and pair counts come back to size
// the next launches).
#include "sim.h"

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

using namespace crk;

#include <atomic>

namespace {
thread_local std::string g_err;
std::atomic<int64_t> g_launches{0};
}

namespace crk {

void note_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
int64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int DBuf::ensure_impl(size_t b)
{
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    size_t nb = std::max<size_t>(b + b / 8, 256);
    cudaError_t e = cudaMalloc(&p, nb);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(CRK_ENOMEM, "cudaMalloc(%zu) failed: %s", nb, cudaGetErrorString(e));
    }
    bytes = nb;
    return CRK_OK;
}

int DBuf::ensure(size_t b)
{
    if (b <= bytes) return CRK_OK;
    return ensure_impl(b);
}

// Grows the buffer keeping its first `keep` bytes (stream-ordered copy).
int DBuf::ensure_keep(size_t b, size_t keep, cudaStream_t st)
{
    if (b <= bytes) return CRK_OK;
    void *old = p;
    size_t nb = std::max<size_t>(b + b / 2, 256);
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, nb);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(CRK_ENOMEM, "cudaMalloc(%zu) failed: %s", nb, cudaGetErrorString(e));
    }
    if (old && keep) {
        e = cudaMemcpyAsync(q, old, std::min(keep, bytes), cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            cudaFree(q);
            return fail(CRK_ECUDA, "buffer growth copy failed: %s", cudaGetErrorString(e));
        }
    }
    if (old) cudaFree(old);
    p = q;
    bytes = nb;
    return CRK_OK;
}

}  // namespace crk

extern "C" const char *crk_last_error(void) { return g_err.c_str(); }

namespace {

size_t rsize(const crk_sim *s) { return s->mixed ? sizeof(float) : sizeof(double); }

void mark(crk_sim *s, int ph, int which)
{
    if (s->timing) {
        cudaEventRecord(s->ev[ph][which], s->st);
        if (which == 1) s->recorded[ph] = true;
    }
}

int alloc_state(DBuf *b, State &s, int64_t n)
{
    size_t nd = (size_t)std::max<int64_t>(n, 1);
    double **dp[13] = {&s.x, &s.y, &s.z, &s.vx, &s.vy, &s.vz, &s.u, &s.m, &s.h, &s.ax, &s.ay, &s.az, &s.du};
    for (int k = 0; k < 13; ++k) {
        RET(b[k].ensure(nd * sizeof(double)));
        *dp[k] = b[k].as<double>();
    }
    RET(b[13].ensure(nd));
    s.species = b[13].as<uint8_t>();
    RET(b[14].ensure(nd * sizeof(uint32_t)));
    s.slot = b[14].as<uint32_t>();
    RET(b[15].ensure(nd * sizeof(uint32_t)));
    s.id = b[15].as<uint32_t>();
    RET(b[16].ensure(nd));
    s.bin = b[16].as<uint8_t>();
    return CRK_OK;
}

// Buffers whose size depends on n only.
int reserve(crk_sim *s, int64_t n)
{
    const size_t nn = (size_t)std::max<int64_t>(n, 1);
    RET(alloc_state(s->stA, s->sa, n));
    RET(alloc_state(s->stB, s->sb, n));
    RET(s->keys.ensure(nn * 8));
    RET(s->keys_alt.ensure(nn * 8));
    RET(s->vals.ensure(nn * 4));
    RET(s->vals_alt.ensure(nn * 4));
    RET(s->counts.ensure(radix_count_words(n) * 4 + 4));
    RET(s->scan_tmp.ensure((scan_tmp_words((int64_t)radix_count_words(n)) + scan_tmp_words(n) + 8) * 4));
    RET(s->flags.ensure(nn * 4));
    RET(s->flag_scan.ensure(nn * 4));
    RET(s->scalars.ensure(64));
    // leaves: at most n
    for (int k = 0; k < 3; ++k) RET(s->lv_u32[k].ensure(nn * 4));
    RET(s->lv_sp.ensure(nn));
    for (int k = 0; k < 3; ++k) RET(s->lv_c[k].ensure(nn * 8));
    for (int k = 0; k < 3; ++k) RET(s->lv_e[k].ensure(nn * 4));
    RET(s->lv_h.ensure(nn * 4));
    s->lv.start = s->lv_u32[0].as<uint32_t>();
    s->lv.count = s->lv_u32[1].as<uint32_t>();
    s->lv.slot = s->lv_u32[2].as<uint32_t>();
    s->lv.species = s->lv_sp.as<uint8_t>();
    s->lv.cx = s->lv_c[0].as<double>();
    s->lv.cy = s->lv_c[1].as<double>();
    s->lv.cz = s->lv_c[2].as<double>();
    s->lv.ex = s->lv_e[0].as<float>();
    s->lv.ey = s->lv_e[1].as<float>();
    s->lv.ez = s->lv_e[2].as<float>();
    s->lv.hmax = s->lv_h.as<float>();
    RET(s->lv_chunk[0].ensure(nn * kChunks * sizeof(float4)));
    RET(s->lv_chunk[1].ensure(nn * kChunks * sizeof(float4)));
    s->lv.clo = s->lv_chunk[0].as<float4>();
    s->lv.chi = s->lv_chunk[1].as<float4>();
    const size_t nnode = 2 * nn + 64;
    for (int k = 0; k < 2; ++k) RET(s->nd_f[k].ensure(nnode * sizeof(float4)));
    RET(s->nd_slot.ensure(nnode * 4));
    s->nd.lo = s->nd_f[0].as<float4>();
    s->nd.hi = s->nd_f[1].as<float4>();
    RET(s->hrow.ensure((nn + 1) * 4));
    RET(s->grow.ensure((nn + 1) * 4));
    RET(s->hcnt.ensure((nn + 1) * 4));
    RET(s->gcnt.ensure((nn + 1) * 4));
    const size_t r4 = 4 * rsize(s);
    RET(s->pm.ensure(nn * r4));
    for (int k = 0; k < 7; ++k) RET(s->hrec[k].ensure(nn * r4));
    RET(s->uhat.ensure(nn * rsize(s)));
    RET(s->acc_h.ensure(nn * r4));
    RET(s->acc_g.ensure(nn * r4));
    if (s->prm.pm_grid > 0) RET(s->acc_pm.ensure(nn * 3 * sizeof(double)));
    RET(s->nbrc.ensure(nn * 4));
    RET(s->nbrh.ensure(nn * 8));
    RET(s->gravc.ensure(nn * 4));
    RET(s->gravh.ensure(nn * 8));
    RET(s->cnt_by_id.ensure(nn * 4));
    RET(s->nl_retry.ensure(16));
    RET(s->census.ensure(32));
    RET(s->err.ensure(16));
    RET(s->nfloor.ensure(16));
    RET(s->partial.ensure((size_t)sums_blocks(n) * 4 * 8 + 64));
    RET(s->sums.ensure(64));
    s->cap_n = std::max<int64_t>(s->cap_n, n);
    return CRK_OK;
}

PassArgs pass_args(crk_sim *s)
{
    PassArgs a{};
    a.n = s->n;
    a.nleaf = s->nleaf;
    a.boxes = s->boxes_d.as<BoxDev>();
    a.s = s->sa;
    a.lv = s->lv;
    a.hrow = s->hrow.as<uint32_t>();
    a.hend = a.hrow ? a.hrow + 1 : nullptr;
    a.hcol = s->hcol.as<uint32_t>();
    a.grow = s->grow.as<uint32_t>();
    a.gend = a.grow ? a.grow + 1 : nullptr;
    a.gcol = s->gcol.as<uint32_t>();
    a.hfr = s->hfr.as<float4>();
    a.gfr = s->gfr.as<float4>();
    a.pm = s->pm.p;
    for (int k = 0; k < 7; ++k) a.hrec[k] = s->hrec[k].p;
    a.uhat = s->uhat.p;
    a.acc_h = s->acc_h.p;
    a.acc_g = s->acc_g.p;
    a.acc_pm = s->prm.pm_grid > 0 && !s->pm_suspend ? s->acc_pm.as<double>() : nullptr;
    a.nbr_count = s->nbrc.as<int32_t>();
    a.nbr_hash = s->nbrh.as<uint64_t>();
    a.grav_count = s->gravc.as<int32_t>();
    a.grav_hash = s->gravh.as<uint64_t>();
    a.err = s->err.as<int>();
    a.nfloor = s->nfloor.as<unsigned long long>();
    a.nl_j = s->nl_j.as<uint32_t>();
    a.hsj = s->hsj.as<uint32_t>();
    a.nl_row = s->nl_row.as<uint32_t>();
    a.nl_len = s->nl_len.as<uint32_t>();
    a.nl_cnt = s->nl_cnt.as<uint32_t>();
    a.ggas = s->grp_gas.as<uint2>();
    a.gall = s->grp_all.as<uint2>();
    a.n_ggas = s->n_ggas;
    a.n_gall = s->n_gall;
    a.bsub = -1;
    a.lmap = nullptr;
    a.nl_bound = 0;
    a.nl_retry = s->nl_retry.as<uint32_t>();
    // each gravity pair once (atomics) when the handle asks for it, except in
    // the service's pool (fixed-order sums) and in a hierarchical substep
    // (rows only for active leaves, so a pair may be seen from one side only)
    a.grav_once = s->mixed && (s->prm.flags & CRK_FLAG_GRAVITY_PAIRS_ONCE) && !s->is_pool && s->bins_bmin < 0;
    a.hydro_once = s->mixed && (s->prm.flags & CRK_FLAG_HYDRO_PAIRS_ONCE) && !s->is_pool && s->bins_bmin < 0;
    return a;
}

int check_physics(const crk_physics &p)
{
    if (!(p.box > 0.0) || !std::isfinite(p.box)) return fail(CRK_EINVAL, "box side must be > 0");
    if (!(p.r_cut > 0.0) || !(p.r_cut < 0.5 * p.box))
        return fail(CRK_EINVAL, "r_cut must satisfy 0 < r_cut < L/2 (got %g, L=%g)", p.r_cut, p.box);
    if (!(p.r_split > 0.0)) return fail(CRK_EINVAL, "r_split must be > 0");
    if (!(p.G >= 0.0) || !std::isfinite(p.G)) return fail(CRK_EINVAL, "G must be finite and >= 0");
    if (!(p.eps_soft >= 0.0)) return fail(CRK_EINVAL, "eps_soft must be >= 0");
    if (!(p.gamma > 1.0)) return fail(CRK_EINVAL, "gamma must be > 1");
    if (!(p.u_floor >= 0.0)) return fail(CRK_EINVAL, "u_floor must be >= 0");
    return CRK_OK;
}

// The short-range factor of the Gaussian split, S(u) = erfc(u) + (2/sqrt(pi))
// u exp(-u^2) with u = r / (2 r_s), has dS/du = -(4/sqrt(pi)) u^2 exp(-u^2)
// and S(0) = 1, so S(u) = 1 - u^3 Q(u^2) with Q(s) = (4/sqrt(pi)) times the
// integral over t in [0, 1] of t^2 exp(-s t^2), an entire function of s.
// Its Taylor coefficients about the middle c of [0, s_max] (s_max the
// square of the box's largest u, at r_cut) are (4/sqrt(pi)) / k! times the
// integral of t^2 (-t^2)^k exp(-c t^2), evaluated here by 48-point
// Gauss-Legendre quadrature (nodes by Newton's method on the Legendre
// recurrence); the series is cut where a term's bound over the range falls
// below 1e-18 of Q's smallest value.  Beyond u = 3 (S < 5e-4) the
// subtraction 1 - u^3 Q would cost more than four digits: erfc is kept.
static void fit_split_series(BoxDev &b)
{
    b.q_deg = 0;
    if (!(b.r_split > 0.0) || !(b.r_cut > 0.0)) return;
    const double umax = b.r_cut / (2.0 * b.r_split);
    if (!(umax <= 3.0)) return;
    const double smax = umax * umax, c = 0.5 * smax, half = 0.5 * smax;
    constexpr int NQ = 48;
    double x[NQ], w[NQ];
    for (int i = 0; i < NQ; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (NQ + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= NQ; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = NQ * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = 0.5 * (z + 1.0);                      // node on [0, 1]
        w[i] = 1.0 / ((1.0 - z * z) * dp * dp);      // half the [-1, 1] weight
    }
    const double norm = 4.0 / std::sqrt(M_PI);
    // smallest Q on the range is at s_max (Q decreases)
    double qmin = 0.0;
    for (int i = 0; i < NQ; ++i) qmin += w[i] * x[i] * x[i] * std::exp(-smax * x[i] * x[i]);
    qmin *= norm;
    double fact = 1.0;
    int deg = 0;
    for (int k = 0; k < kSplitTerms; ++k) {
        if (k > 0) fact *= k;
        double sum = 0.0;
        for (int i = 0; i < NQ; ++i) {
            const double t2 = x[i] * x[i];
            sum += w[i] * t2 * std::pow(-t2, k) * std::exp(-c * t2);
        }
        b.q_coef[k] = norm * sum / fact;
        deg = k + 1;
        if (std::fabs(b.q_coef[k]) * std::pow(half, k) < 1e-18 * qmin && k >= 4) break;
    }
    if (std::fabs(b.q_coef[deg - 1]) * std::pow(half, deg - 1) >= 1e-16 * qmin) return;  // series too long
    b.q_deg = deg;
    b.q_c = c;
    b.q_inv4rs2 = 1.0 / (4.0 * b.r_split * b.r_split);
}

BoxDev box_dev(const crk_physics &p)
{
    BoxDev b{};
    b.L = p.box;
    b.halfL = 0.5 * p.box;
    b.G = p.G;
    b.gamma = p.gamma;
    b.r_cut = p.r_cut;
    b.r_split = p.r_split;
    b.eps_soft = p.eps_soft;
    b.av_alpha = p.av_alpha;
    b.av_beta = p.av_beta;
    b.av_eps2 = p.av_eps2;
    b.u_floor = p.u_floor;
    b.dt = 0.0;
    b.hdt = 0.0;
    b.cm_shift = 63;
    b.active = 1;
    fit_split_series(b);
    return b;
}

// Chaining-mesh level of a box: the Morton level b (2^b bins per side) that
// gives about four leaves of each species per bin, the paper's coarse bins
// (Sec. IV-B1) sized to the leaf capacity.
int auto_cm_level(int64_t n_species, int cap)
{
    double per_side = std::cbrt((double)std::max<int64_t>(n_species, 1) / (4.0 * cap));
    int b = (int)std::floor(std::log2(std::max(per_side, 1.0)));
    return std::min(std::max(b, 0), 10);
}

int upload_boxes(crk_sim *s)
{
    RET(s->boxes_d.ensure(std::max<size_t>(s->boxes.size(), 1) * sizeof(BoxDev)));
    CK(cudaMemcpyAsync(s->boxes_d.p, s->boxes.data(), s->boxes.size() * sizeof(BoxDev),
                       cudaMemcpyHostToDevice, s->st));
    return CRK_OK;
}

// A host synchronisation inside a step (counted: a step captured as a graph
// has none).
#define HOST_SYNC(s)                         \
    do {                                     \
        ++(s)->host_syncs;                   \
        CK(cudaStreamSynchronize((s)->st));  \
    } while (0)

int read_error(crk_sim *s)
{
    CK(cudaMemcpyAsync(s->host_err, s->err.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, s->st));
    HOST_SYNC(s);
    const int code = s->host_err[0], idx = s->host_err[1];
    if (code == CRK_ESINGULAR)
        return fail(CRK_ESINGULAR, "second-moment matrix of gas particle %d is singular", idx);
    if (code == CRK_ETIMEOUT)
        return fail(CRK_ETIMEOUT, "a bounded retry loop ran out (particle %d)", idx);
    if (code == CRK_EINVAL)
        return fail(CRK_EINVAL, "particle %d is invalid (position outside [0,L), non-finite value, "
                                "mass <= 0, or gas h with 2h <= 0 or 2h >= L/2)", idx);
    if (code != 0) return fail(code, "device error %d at particle %d", code, idx);
    return CRK_OK;
}

int reset_error(crk_sim *s)
{
    int init[2] = {0, 0x7fffffff};
    CK(cudaMemcpyAsync(s->err.p, init, sizeof init, cudaMemcpyHostToDevice, s->st));
    return CRK_OK;
}

// Tree build (S1) and leaf-pair lists (S2).  mode 0: sort every
// rebuild_every-th call; 1: sort now; 2: keep the leaves while they are valid.
enum { TREE_RULE = 0, TREE_SORT = 1, TREE_KEEP = 2 };
int build_tree(crk_sim *s, int mode = TREE_RULE)
{
    const int64_t n = s->n;
    cudaStream_t st = s->st;
    mark(s, PH_TREE, 0);
    uint32_t *tmp = s->scan_tmp.as<uint32_t>();
    uint32_t *sc = s->scalars.as<uint32_t>();
    // Between rebuilds the leaves keep their particles and their boxes grow
    // with the particles (paper Sec. IV-B1): no sort, only new bounds, node
    // boxes and pair lists.  Added or removed particles force a rebuild.
    const int every = std::max(s->prm.rebuild_every, 1);
    bool reuse = s->tree_valid && s->n_dead == 0 && s->since_rebuild + 1 < every;
    if (mode == TREE_SORT) reuse = false;
    else if (mode == TREE_KEEP) reuse = s->tree_valid && s->n_dead == 0;
    if (reuse) {
        ++s->since_rebuild;
    } else {
        launch_morton_keys(s->sa, s->boxes_d.as<BoxDev>(), n, s->slot_bits, s->keys.as<uint64_t>(),
                           s->vals.as<uint32_t>(), st);
        // One box: sort the key bits down to sort_levels octree levels below
        // the chaining-mesh bin (the leaves of the last sort used fewer; the
        // order inside a leaf comes from the k-d pass): 3-5 radix passes
        // instead of 8.  Several boxes sort every bit, so that a box's leaves
        // and their order never depend on the other boxes (the service's
        // alone-equals-in-the-mix guarantee).
        int first_bit = 0;
        if (s->slot_bits == 0 && s->nbox == 1)
            first_bit = std::max(s->boxes[0].cm_shift - 3 * s->sort_levels, 0);
        uint64_t *ko;
        uint32_t *vo;
        radix_sort_u64(s->keys.as<uint64_t>(), s->vals.as<uint32_t>(), s->keys_alt.as<uint64_t>(),
                       s->vals_alt.as<uint32_t>(), n, s->counts.as<uint32_t>(), tmp, first_bit, 64, st, &ko,
                       &vo);
        // particles of removed pool slots carry the largest key and sort last
        const int64_t nlive = n - s->n_dead;
        CK(cudaMemsetAsync(sc + 12, 0, 2 * sizeof(uint32_t), st));
        launch_leaf_flags(ko, s->slot_bits, s->boxes_d.as<BoxDev>(), nlive, s->cap, s->flags.as<uint32_t>(),
                          first_bit, sc + 12, st);
        scan_exclusive_u32(s->flags.as<uint32_t>(), s->flag_scan.as<uint32_t>(), nlive, sc + 0, tmp, st);
        CK(cudaMemcpyAsync(s->host_scalars, sc, 14 * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        HOST_SYNC(s);
        s->nleaf = (int)s->host_scalars[0];
        if (s->nleaf >= (1 << 26))  // the leaf-pair walk packs leaf indices into 26 bits
            return fail(CRK_EOVERFLOW, "%d leaves: at most 2^26 - 1", s->nleaf);
        // the next sort: two levels below the deepest leaf of this one, or all
        // levels when a cell had to be cut by count above unsorted levels
        s->sort_levels = s->host_scalars[13] ? kAllLevels : std::min(kAllLevels, (int)s->host_scalars[12] + 2);
        launch_leaf_setup(s->flags.as<uint32_t>(), s->flag_scan.as<uint32_t>(), nlive, s->nleaf, s->lv, st);
        // k-d order inside every leaf (on the unsorted state through the sort's
        // permutation), then one gather of the whole state
        launch_leaf_kd_order(s->sa, s->lv, s->nleaf, vo, st);
        launch_permute(s->sa, s->sb, vo, n, st);
        std::swap(s->sa, s->sb);
        for (int k = 0; k < 17; ++k) std::swap(s->stA[k], s->stB[k]);
        s->n = nlive;
        s->n_dead = 0;
        s->since_rebuild = 0;
        s->tree_valid = true;
    }
    launch_leaf_bounds(s->sa, s->boxes_d.as<BoxDev>(), s->lv, s->nleaf, s->mixed ? 1 : 0, s->pm.p,
                       s->nd, st);
    mark(s, PH_TREE, 1);
    mark(s, PH_PAIRS, 0);
    launch_build_nodes(s->nd, s->nleaf, st);
    const BoxDev *bd = s->boxes_d.as<BoxDev>();
    // hierarchical substeps: only the leaves holding an active particle need
    // gravity rows (the hydro rows of every gas leaf feed the active sets)
    const uint8_t *gmask = nullptr;
    if (s->bins_bmin >= 0) {
        RET(s->bflag.ensure(3 * (size_t)std::max(s->nleaf, 1)));
        launch_leaf_active(s->lv, s->nleaf, s->sa.bin, s->bins_bmin, s->bflag.as<uint8_t>(), st);
        gmask = s->bflag.as<uint8_t>();
    }
    // one walk per list into rows of fixed capacity, packed after the scan;
    // a leaf with more pairs than that makes both lists walk twice (count,
    // fill), and the next 16 builds walk twice from the start
    const size_t nls = (size_t)std::max(s->nleaf, 1);
    const bool scratch = s->pair_two_pass_left == 0;
    uint32_t *scol_h = nullptr, *scol_g = nullptr;
    float4 *sfr_h = nullptr, *sfr_g = nullptr;
    CK(cudaMemsetAsync(sc + 7, 0, sizeof(uint32_t), st));
    if (scratch) {
        RET(s->pscr_col.ensure(nls * (kPairCapH + kPairCapG) * sizeof(uint32_t)));
        RET(s->pscr_fr.ensure(nls * (kPairCapH + kPairCapG) * sizeof(float4)));
        RET(s->pscr_st.ensure(nls * kPairCapH * sizeof(uint32_t)));
        scol_h = s->pscr_col.as<uint32_t>();
        scol_g = scol_h + nls * kPairCapH;
        sfr_h = s->pscr_fr.as<float4>();
        sfr_g = sfr_h + nls * kPairCapH;
        launch_pair_scratch(s->nd, s->lv, bd, s->nleaf, 1, s->hcnt.as<uint32_t>(), kPairCapH, scol_h, sfr_h,
                            s->pscr_st.as<uint32_t>(), sc + 7, st);
        launch_pair_scratch(s->nd, s->lv, bd, s->nleaf, 0, s->gcnt.as<uint32_t>(), kPairCapG, scol_g, sfr_g,
                            nullptr, sc + 7, st, gmask);
    } else {
        --s->pair_two_pass_left;
        launch_pair_count(s->nd, s->lv, bd, s->nleaf, 1, s->hcnt.as<uint32_t>(), st);
        launch_pair_count(s->nd, s->lv, bd, s->nleaf, 0, s->gcnt.as<uint32_t>(), st, gmask);
    }
    scan_exclusive_u32(s->hcnt.as<uint32_t>(), s->hrow.as<uint32_t>(), s->nleaf, sc + 1, tmp, st);
    scan_exclusive_u32(s->gcnt.as<uint32_t>(), s->grow.as<uint32_t>(), s->nleaf, sc + 2, tmp, st);
    // warp work items: gas-leaf groups, then all-leaf groups
    RET(s->grp_cnt.ensure((size_t)std::max(s->nleaf, 1) * 4 * 2));
    RET(s->grp_off.ensure((size_t)std::max(s->nleaf, 1) * 4 * 2));
    uint32_t *gc = s->grp_cnt.as<uint32_t>(), *go = s->grp_off.as<uint32_t>();
    const size_t nl = (size_t)std::max(s->nleaf, 1);
    launch_group_count(s->lv, s->nleaf, 1, gc, st);
    launch_group_count(s->lv, s->nleaf, 0, gc + nl, st);
    scan_exclusive_u32(gc, go, s->nleaf, sc + 3, tmp, st);
    scan_exclusive_u32(gc + nl, go + nl, s->nleaf, sc + 4, tmp, st);
    CK(cudaMemcpyAsync(s->host_scalars + 1, sc + 1, 7 * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    HOST_SYNC(s);
    const bool pair_overflow = !scratch || s->host_scalars[7] != 0;
    if (scratch && pair_overflow) s->pair_two_pass_left = 16;
    s->npair_h = s->host_scalars[1];
    s->npair_g = s->host_scalars[2];
    s->n_ggas = s->host_scalars[3];
    s->n_gall = s->host_scalars[4];
    RET(s->grp_gas.ensure((size_t)std::max<uint32_t>(s->n_ggas, 1) * sizeof(uint2)));
    RET(s->grp_all.ensure((size_t)std::max<uint32_t>(s->n_gall, 1) * sizeof(uint2)));
    launch_group_fill(s->lv, s->nleaf, 1, go, s->grp_gas.as<uint2>(), st);
    launch_group_fill(s->lv, s->nleaf, 0, go + nl, s->grp_all.as<uint2>(), st);
    // row[nleaf] = total
    CK(cudaMemcpyAsync(s->hrow.as<uint32_t>() + s->nleaf, sc + 1, 4, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(s->grow.as<uint32_t>() + s->nleaf, sc + 2, 4, cudaMemcpyDeviceToDevice, st));
    RET(s->hcol.ensure((size_t)std::max<int64_t>(s->npair_h, 1) * 4));
    RET(s->gcol.ensure((size_t)std::max<int64_t>(s->npair_g, 1) * 4));
    RET(s->hfr.ensure((size_t)std::max<int64_t>(s->npair_h, 1) * 16));
    RET(s->hsj.ensure((size_t)std::max<int64_t>(s->npair_h, 1) * 4));
    RET(s->gfr.ensure((size_t)std::max<int64_t>(s->npair_g, 1) * 16));
    if (pair_overflow) {
        launch_pair_fill(s->nd, s->lv, bd, s->nleaf, 1, s->hrow.as<uint32_t>(), s->hcol.as<uint32_t>(),
                         s->hfr.as<float4>(), s->hsj.as<uint32_t>(), st);
        launch_pair_fill(s->nd, s->lv, bd, s->nleaf, 0, s->grow.as<uint32_t>(), s->gcol.as<uint32_t>(),
                         s->gfr.as<float4>(), nullptr, st, gmask);
    } else {
        launch_pair_compact(s->nleaf, kPairCapH, s->hcnt.as<uint32_t>(), s->hrow.as<uint32_t>(), scol_h, sfr_h,
                            s->pscr_st.as<uint32_t>(), s->hcol.as<uint32_t>(), s->hfr.as<float4>(),
                            s->hsj.as<uint32_t>(), st);
        launch_pair_compact(s->nleaf, kPairCapG, s->gcnt.as<uint32_t>(), s->grow.as<uint32_t>(), scol_g, sfr_g,
                            nullptr, s->gcol.as<uint32_t>(), s->gfr.as<float4>(), nullptr, st);
    }
    mark(s, PH_PAIRS, 1);
    return CRK_OK;
}

// Sizes the hydro neighbour lists: every group's row count, from a count
// pass over the candidates, or (use_bounds) from the previous step's list
// sizes with a margin; row offsets by a scan, then the list storage (one
// synchronisation for the total).
static int size_hydro_lists(crk_sim *s, PassArgs &a, bool want_counts, bool use_bounds = false)
{
    cudaStream_t st = s->st;
    if (a.n_ggas == 0) {
        s->nl_rows = 0;
        return CRK_OK;
    }
    const size_t ng = (size_t)a.n_ggas;
    RET(s->nl_cnt.ensure((size_t)std::max<int64_t>(s->n, 1) * 4));
    RET(s->nl_len.ensure(ng * 4));
    RET(s->nl_row.ensure(ng * 4));
    a.nl_cnt = s->nl_cnt.as<uint32_t>();
    a.nl_len = s->nl_len.as<uint32_t>();
    a.nl_row = s->nl_row.as<uint32_t>();
    a.nl_bound = use_bounds ? 1 : 0;
    if (use_bounds) {
        launch_hlist_bound(a, s->cnt_by_id.as<uint32_t>(), st);
        CK(cudaMemsetAsync(a.nl_retry, 0, sizeof(uint32_t), st));
    } else {
        launch_hlist_count(a, s->mixed ? 1 : 0, s->cap, want_counts, st);
    }
    uint32_t *sc = s->scalars.as<uint32_t>();
    scan_exclusive_u32(a.nl_len, a.nl_row, a.n_ggas, sc + 5, s->scan_tmp.as<uint32_t>(), st);
    CK(cudaMemcpyAsync(s->host_scalars + 5, sc + 5, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    HOST_SYNC(s);
    s->nl_rows = s->host_scalars[5];
    const size_t entries = (size_t)std::max<int64_t>(s->nl_rows, 1) * 32u;
    RET(s->nl_j.ensure(entries * 4));
    a.nl_j = s->nl_j.as<uint32_t>();
    return CRK_OK;
}

// Lists and density of the gas groups of a: rows sized from the last step's
// counts when they are known (a list that outgrows them is counted and
// filled again), the fill, the density evaluation, and the counts kept for
// the next step.
static int density_pass(crk_sim *s, PassArgs &a, bool want_counts)
{
    cudaStream_t st = s->st;
    const int mixed = s->mixed ? 1 : 0;
    RET(size_hydro_lists(s, a, want_counts, s->cnt_valid && !s->is_pool));
    if (a.census) CK(cudaMemsetAsync(a.census, 0, 2 * sizeof(unsigned long long), st));
    launch_hlist_fill(a, mixed, s->cap, want_counts, st);
    if (a.nl_bound) {
        CK(cudaMemcpyAsync(s->host_scalars + 6, a.nl_retry, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        HOST_SYNC(s);
        if (s->host_scalars[6]) {
            RET(size_hydro_lists(s, a, want_counts, false));
            if (a.census) CK(cudaMemsetAsync(a.census, 0, 2 * sizeof(unsigned long long), st));
            launch_hlist_fill(a, mixed, s->cap, want_counts, st);
        }
    }
    // without neighbour counts the fill pass has formed the density already
    if (want_counts) launch_density_eval(a, mixed, s->cap, want_counts, st);
    if (!s->is_pool) launch_keep_counts(a, s->cnt_by_id.as<uint32_t>(), st);
    return CRK_OK;
}

// One step.  kdk = false: a force evaluation at the current state (dt = 0).
int run_step(crk_sim *s, const double *dt_per_box, bool want_counts)
{
    cudaStream_t st = s->st;
    for (int b = 0; b < s->nbox; ++b) {
        const double dt = dt_per_box ? dt_per_box[b] : 0.0;
        s->boxes[b].dt = dt;
        s->boxes[b].hdt = 0.5 * dt;
    }
    RET(upload_boxes(s));
    RET(reset_error(s));
    if (s->timing) cudaEventRecord(s->ev_all[0], st);
    for (bool &r : s->recorded) r = false;
    const int64_t launches0 = launches_so_far();
    if (dt_per_box) {
        mark(s, PH_KICK, 0);
        launch_kick_drift(s->sa, s->boxes_d.as<BoxDev>(), s->n, s->nfloor.as<unsigned long long>(), st);
        mark(s, PH_KICK, 1);
    }
    RET(build_tree(s));
    if (s->prm.pm_grid > 0 && !s->pm_suspend) {
        mark(s, PH_PM, 0);
        RET(pm_accelerations(s, s->acc_pm.as<double>(), false));
        mark(s, PH_PM, 1);
    }
    PassArgs a = pass_args(s);
    if (!want_counts) {
        a.nbr_count = nullptr;
        a.nbr_hash = nullptr;
        a.grav_count = nullptr;
        a.grav_hash = nullptr;
    } else {
        a.census = s->census.as<unsigned long long>();
        CK(cudaMemsetAsync(a.census, 0, 4 * sizeof(unsigned long long), st));
    }
    const int mixed = s->mixed ? 1 : 0;
    mark(s, PH_D, 0);
    launch_records(a, mixed, st);
    RET(density_pass(s, a, want_counts));
    if (!s->is_pool) s->cnt_valid = true;
    mark(s, PH_D, 1);
    mark(s, PH_M, 0);
    launch_moments(a, mixed, s->cap, st);
    mark(s, PH_M, 1);
    mark(s, PH_H, 0);
    launch_hydro(a, mixed, s->cap, st);
    mark(s, PH_H, 1);
    mark(s, PH_G, 0);
    launch_gravity(a, mixed, s->cap, want_counts, st);
    mark(s, PH_G, 1);
    mark(s, PH_KDK, 0);
    launch_final_kick(a, mixed, s->nfloor.as<unsigned long long>(), st);
    mark(s, PH_KDK, 1);
    if (s->timing) cudaEventRecord(s->ev_all[1], st);
    CK(cudaGetLastError());
    RET(read_error(s));
    if (a.census) {  // read_error has synchronised the stream: the counters are final
        CK(cudaMemcpy(s->census_h, a.census, sizeof(s->census_h), cudaMemcpyDeviceToHost));
        s->census_rows = s->nl_rows;
    }
    if (s->timing) {
        for (int ph = 0; ph < PH_N; ++ph) {
            if (!s->recorded[ph]) continue;
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, s->ev[ph][0], s->ev[ph][1]) == cudaSuccess) s->acc_ms[ph] += ms;
            else cudaGetLastError();
        }
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, s->ev_all[0], s->ev_all[1]) == cudaSuccess) s->total_ms += ms;
        else cudaGetLastError();
        s->calls++;
        s->launches += launches_so_far() - launches0;
    }
    s->have_forces = true;
    if (dt_per_box) ++s->steps_run;
    return CRK_OK;
}

int copy_in(crk_sim *s, void *dst, const void *src, size_t bytes, int mem)
{
    if (bytes == 0) return CRK_OK;
    CK(cudaMemcpyAsync(dst, src, bytes,
                       mem == CRK_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->st));
    return CRK_OK;
}

int load_impl(crk_sim *s, int nbox, const int64_t *counts, const crk_physics *phys,
              const double *pos, const double *vel, const double *mass, const double *u,
              const double *h, const uint8_t *species, int mem)
{
    if (nbox < 1) return fail(CRK_EINVAL, "nbox must be >= 1");
    if (nbox > 1 && s->prm.pm_grid > 0) return fail(CRK_EINVAL, "a mesh (pm_grid > 0) needs one box");
    if (mem != CRK_MEM_HOST && mem != CRK_MEM_DEVICE) return fail(CRK_EINVAL, "bad mem flag");
    int64_t n = 0;
    for (int b = 0; b < nbox; ++b) {
        if (counts[b] < 0) return fail(CRK_EINVAL, "negative particle count in box %d", b);
        RET(check_physics(phys[b]));
        n += counts[b];
    }
    if (n > 0 && (!pos || !vel || !mass || !u || !h || !species))
        return fail(CRK_EINVAL, "null input array");
    if (n >= (int64_t)1 << 31) return fail(CRK_EINVAL, "at most 2^31 - 1 particles");
    CK(cudaSetDevice(s->device));
    RET(reserve(s, n));
    s->n = n;
    s->tree_valid = false;
    s->cnt_valid = false;
    s->nbox = nbox;
    int sb = 0;
    while ((1 << sb) < nbox) ++sb;
    s->slot_bits = sb;
    s->boxes.assign(nbox, BoxDev{});
    s->box_count.assign(counts, counts + nbox);
    // species counts per box for the chaining-mesh level (host arrays or a copy)
    std::vector<uint8_t> sp_host;
    const uint8_t *sp = species;
    if (mem == CRK_MEM_DEVICE && n > 0) {
        sp_host.resize((size_t)n);
        CK(cudaMemcpy(sp_host.data(), species, (size_t)n, cudaMemcpyDeviceToHost));
        sp = sp_host.data();
    }
    std::vector<uint32_t> slot_of((size_t)std::max<int64_t>(n, 1));
    int64_t off = 0;
    for (int b = 0; b < nbox; ++b) {
        int64_t ng = 0;
        for (int64_t k = off; k < off + counts[b]; ++k) {
            slot_of[(size_t)k] = (uint32_t)b;
            ng += sp[k] == CRK_GAS;
        }
        const int64_t ns = std::max(ng, counts[b] - ng);
        int lvl = s->prm.cm_level > 0 ? s->prm.cm_level : auto_cm_level(ns, s->cap);
        lvl = std::min(lvl, (63 - sb) / 3);
        s->boxes[b] = box_dev(phys[b]);
        s->boxes[b].cm_shift = 63 - sb - 3 * lvl;
        off += counts[b];
    }
    RET(upload_boxes(s));
    // Stage inputs on the device, then scatter into the SoA state.
    const size_t nn = (size_t)n;
    const size_t need = nn * (3 + 3 + 1 + 1 + 1) * sizeof(double) + nn + nn * 4 + 64;
    RET(s->in_stage.ensure(need));
    char *base = s->in_stage.as<char>();
    double *d_pos = (double *)base;
    double *d_vel = d_pos + 3 * nn;
    double *d_mass = d_vel + 3 * nn;
    double *d_u = d_mass + nn;
    double *d_h = d_u + nn;
    uint32_t *d_slot = (uint32_t *)(d_h + nn);
    uint8_t *d_sp = (uint8_t *)(d_slot + nn);
    RET(copy_in(s, d_pos, pos, 3 * nn * 8, mem));
    RET(copy_in(s, d_vel, vel, 3 * nn * 8, mem));
    RET(copy_in(s, d_mass, mass, nn * 8, mem));
    RET(copy_in(s, d_u, u, nn * 8, mem));
    RET(copy_in(s, d_h, h, nn * 8, mem));
    RET(copy_in(s, d_sp, species, nn, mem));
    if (n > 0) CK(cudaMemcpyAsync(d_slot, slot_of.data(), nn * 4, cudaMemcpyHostToDevice, s->st));
    launch_load_state(s->sa, n, d_pos, d_vel, d_mass, d_u, d_h, d_sp, d_slot, s->st);
    RET(reset_error(s));
    launch_validate(s->sa, s->boxes_d.as<BoxDev>(), n, s->err.as<int>(), s->st);
    CK(cudaMemsetAsync(s->nfloor.p, 0, 8, s->st));
    CK(cudaGetLastError());
    int rc = read_error(s);
    if (rc != CRK_OK) {
        s->n = 0;
        s->tree_valid = false;
        return rc;
    }
    s->have_forces = false;
    return CRK_OK;
}

template <typename T>
int deliver(crk_sim *s, T *user, size_t count, int mem, T **dev_target, size_t &stage_off)
{
    // Where the un-permute kernel writes: the user's device buffer directly,
    // or a slice of the staging buffer for host outputs.
    if (!user) {
        *dev_target = nullptr;
        return CRK_OK;
    }
    if (mem == CRK_MEM_DEVICE) {
        *dev_target = user;
        return CRK_OK;
    }
    *dev_target = reinterpret_cast<T *>(s->staging.as<char>() + stage_off);
    stage_off += (count * sizeof(T) + 255) & ~size_t(255);
    return CRK_OK;
}

}  // namespace

extern "C" int crk_create(const crk_params *params, void *cuda_stream, crk_sim **out)
{
    if (!params || !out) return fail(CRK_EINVAL, "null argument");
    if (params->leaf_cap != 32 && params->leaf_cap != 64 && params->leaf_cap != 128)
        return fail(CRK_EINVAL, "leaf_cap must be 32, 64 or 128 (got %d)", params->leaf_cap);
    if (params->precision != CRK_FP64 && params->precision != CRK_MIXED)
        return fail(CRK_EINVAL, "precision must be CRK_FP64 or CRK_MIXED");
    if (params->kernel != CRK_WENDLAND_C4) return fail(CRK_EINVAL, "unsupported kernel");
    if (params->cm_level < 0 || params->cm_level > 10) return fail(CRK_EINVAL, "cm_level in [0, 10]");
    if (params->rebuild_every < 0) return fail(CRK_EINVAL, "rebuild_every must be >= 0");
    if (params->flags & ~(CRK_FLAG_GRAVITY_PAIRS_ONCE | CRK_FLAG_NO_GRAPH | CRK_FLAG_HYDRO_PAIRS_ONCE))
        return fail(CRK_EINVAL, "unknown flags bits 0x%x", params->flags);
    if (params->graph_margin_pct < 0 || params->graph_margin_pct > 1000)
        return fail(CRK_EINVAL, "graph_margin_pct must be in [0, 1000]");
    if (params->pm_grid != 0 && (params->pm_grid < 4 || params->pm_grid > 1024 || params->pm_grid % 2))
        return fail(CRK_EINVAL, "pm_grid must be 0 or an even number in [4, 1024] (got %d)", params->pm_grid);
    crk_sim *s = new crk_sim();
    s->prm = *params;
    s->mixed = params->precision == CRK_MIXED;
    s->cap = params->leaf_cap;
    s->ds_margin = 1.0 + (params->graph_margin_pct > 0 ? params->graph_margin_pct : 25) / 100.0;
    s->st = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaMallocHost(&s->host_scalars, 64);
    if (e == cudaSuccess) e = cudaMallocHost(&s->host_err, 64);
    if (e != cudaSuccess) {
        int code = fail(CRK_ECUDA, "CUDA initialisation failed: %s", cudaGetErrorString(e));
        cudaGetLastError();
        delete s;
        return code;
    }
    for (int ph = 0; ph < PH_N; ++ph)
        for (int w = 0; w < 2; ++w) cudaEventCreate(&s->ev[ph][w]);
    cudaEventCreate(&s->ev_all[0]);
    cudaEventCreate(&s->ev_all[1]);
    *out = s;
    return CRK_OK;
}

extern "C" int crk_load(crk_sim *sim, int64_t n, const double *pos, const double *vel,
                        const double *mass, const double *u, const double *h,
                        const uint8_t *species, int mem)
{
    if (!sim) return fail(CRK_EINVAL, "null handle");
    if (n < 0) return fail(CRK_EINVAL, "n must be >= 0");
    return load_impl(sim, 1, &n, &sim->prm.phys, pos, vel, mass, u, h, species, mem);
}

extern "C" int crk_load_boxes(crk_sim *sim, int nbox, const int64_t *counts,
                              const crk_physics *phys, const double *pos, const double *vel,
                              const double *mass, const double *u, const double *h,
                              const uint8_t *species, int mem)
{
    if (!sim || !counts || !phys) return fail(CRK_EINVAL, "null argument");
    return load_impl(sim, nbox, counts, phys, pos, vel, mass, u, h, species, mem);
}

extern "C" int crk_forces(crk_sim *s, crk_outputs *out)
{
    if (!s || !out) return fail(CRK_EINVAL, "null argument");
    if (out->mem != CRK_MEM_HOST && out->mem != CRK_MEM_DEVICE) return fail(CRK_EINVAL, "bad mem flag");
    CK(cudaSetDevice(s->device));
    const bool counts = out->nbr_count || out->nbr_hash || out->grav_count || out->grav_hash;
    RET(run_step(s, nullptr, counts));
    PassArgs a = pass_args(s);
    if (!counts) {
        a.nbr_count = nullptr;
        a.nbr_hash = nullptr;
        a.grav_count = nullptr;
        a.grav_hash = nullptr;
    }
    const size_t n = (size_t)s->n;
    if (out->mem == CRK_MEM_HOST) RET(s->staging.ensure(std::max<size_t>(n, 1) * 8 * 24 + 4096));
    size_t off = 0;
    double *acc, *dudt, *rho, *A, *B, *gA, *gB;
    int32_t *nc, *gc;
    uint64_t *nh, *gh;
    RET(deliver(s, out->acc, 3 * n, out->mem, &acc, off));
    RET(deliver(s, out->dudt, n, out->mem, &dudt, off));
    RET(deliver(s, out->rho, n, out->mem, &rho, off));
    RET(deliver(s, out->A, n, out->mem, &A, off));
    RET(deliver(s, out->B, 3 * n, out->mem, &B, off));
    RET(deliver(s, out->gradA, 3 * n, out->mem, &gA, off));
    RET(deliver(s, out->gradB, 9 * n, out->mem, &gB, off));
    RET(deliver(s, out->nbr_count, n, out->mem, &nc, off));
    RET(deliver(s, out->nbr_hash, n, out->mem, &nh, off));
    RET(deliver(s, out->grav_count, n, out->mem, &gc, off));
    RET(deliver(s, out->grav_hash, n, out->mem, &gh, off));
    launch_unpermute_outputs(a, s->mixed ? 1 : 0, acc, dudt, rho, A, B, gA, gB, nc, nh, gc, gh, s->st);
    if (out->mem == CRK_MEM_HOST && n > 0) {
        struct { void *u; const void *d; size_t b; } cp[] = {
            {out->acc, acc, 3 * n * 8}, {out->dudt, dudt, n * 8}, {out->rho, rho, n * 8},
            {out->A, A, n * 8}, {out->B, B, 3 * n * 8}, {out->gradA, gA, 3 * n * 8},
            {out->gradB, gB, 9 * n * 8}, {out->nbr_count, nc, n * 4}, {out->nbr_hash, nh, n * 8},
            {out->grav_count, gc, n * 4}, {out->grav_hash, gh, n * 8}};
        for (auto &c : cp)
            if (c.u) CK(cudaMemcpyAsync(c.u, c.d, c.b, cudaMemcpyDeviceToHost, s->st));
    }
    launch_rate_sums(a, s->mixed ? 1 : 0, s->partial.as<double>(), sums_blocks(s->n), s->sums.as<double>(), s->st);
    double sums[4];
    CK(cudaMemcpyAsync(sums, s->sums.p, sizeof sums, cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    out->momentum_rate[0] = sums[0];
    out->momentum_rate[1] = sums[1];
    out->momentum_rate[2] = sums[2];
    out->energy_rate = sums[3];
    return CRK_OK;
}

// ------------------------------------------------------- graph-captured steps
// A KDK step with every size kept on the device: leaves, leaf pairs, target
// groups and list rows are counted by scans into the device sizes block and
// every launch after them is sized by a capacity fixed on the host (from the
// last host-sized step, with a margin) and reads the true count on the
// device; the pass kernels are persistent launches that drain a device work
// queue of (leaf, target group) items of every box.  The leaf-pair lists are
// walked twice (count, fill at scanned offsets), hydro list rows are sized
// from the last step's counts.  Nothing is read back, so the step can
// be captured into a CUDA graph; an overflow of a capacity is recorded on the
// device (and zeroes the counts the rest of the step launches over).
static int run_step_ds(crk_sim *s)
{
    cudaStream_t st = s->st;
    const int64_t n = s->n;
    const int mixed = s->mixed ? 1 : 0;
    const BoxDev *bd = s->boxes_d.as<BoxDev>();
    uint32_t *dz = s->dz.as<uint32_t>();
    uint32_t *tmp = s->scan_tmp.as<uint32_t>();
    const int capL = s->ds_cap_leaf;
    const size_t nl = (size_t)capL;
    const uint32_t capI = s->ds_cap_items;
    CK(cudaMemsetAsync(dz + DZ_QUEUE, 0, kQueueSlots * sizeof(uint32_t), st));
    launch_kick_drift(s->sa, bd, n, s->nfloor.as<unsigned long long>(), st);
    // S1: keys, sort (the bits the last host-sized sort chose), leaves
    launch_morton_keys(s->sa, bd, n, s->slot_bits, s->keys.as<uint64_t>(), s->vals.as<uint32_t>(), st);
    int first_bit = 0;
    if (s->slot_bits == 0 && s->nbox == 1) first_bit = std::max(s->boxes[0].cm_shift - 3 * s->sort_levels, 0);
    uint64_t *ko;
    uint32_t *vo;
    radix_sort_u64(s->keys.as<uint64_t>(), s->vals.as<uint32_t>(), s->keys_alt.as<uint64_t>(),
                   s->vals_alt.as<uint32_t>(), n, s->counts.as<uint32_t>(), tmp, first_bit, 64, st, &ko, &vo);
    launch_leaf_flags(ko, s->slot_bits, bd, n, s->cap, s->flags.as<uint32_t>(), first_bit, dz + DZ_STATS, st);
    scan_exclusive_u32(s->flags.as<uint32_t>(), s->flag_scan.as<uint32_t>(), n, dz + DZ_NLEAF_RAW, tmp, st);
    launch_ds_check(dz, 0, (uint32_t)capL, nullptr, st);
    const uint32_t *nld = dz + DZ_NLEAF;
    launch_leaf_setup(s->flags.as<uint32_t>(), s->flag_scan.as<uint32_t>(), n, capL, s->lv, st, nld);
    launch_leaf_kd_order(s->sa, s->lv, capL, vo, st, nld);
    launch_permute(s->sa, s->sb, vo, n, st);
    std::swap(s->sa, s->sb);
    for (int k = 0; k < 17; ++k) std::swap(s->stA[k], s->stB[k]);
    launch_leaf_bounds(s->sa, bd, s->lv, capL, mixed, s->pm.p, s->nd, st, nld);
    // S2: hierarchy over the capacity; each list walked twice (count, then
    // fill into CSR rows from a scan whose total is checked on the device)
    Nodes nd = s->nd;
    launch_build_nodes(nd, capL, st);
    uint32_t *hrow = s->hrow.as<uint32_t>(), *grow = s->grow.as<uint32_t>();
    uint32_t *hc = s->hcnt.as<uint32_t>(), *gcn = s->gcnt.as<uint32_t>();
    if (s->ds_one_walk) {
        // one walk into rows of fixed capacity (the first step's rows fitted),
        // packed after the scan; a row that does not fit is an overflow
        uint32_t *scol_h = s->pscr_col.as<uint32_t>(), *scol_g = scol_h + nl * kPairCapH;
        float4 *sfr_h = s->pscr_fr.as<float4>(), *sfr_g = sfr_h + nl * kPairCapH;
        CK(cudaMemsetAsync(dz + DZ_ROW_OVF, 0, sizeof(uint32_t), st));
        launch_pair_scratch(nd, s->lv, bd, capL, 1, hc, kPairCapH, scol_h, sfr_h, s->pscr_st.as<uint32_t>(),
                            dz + DZ_ROW_OVF, st, nullptr, nld);
        launch_pair_scratch(nd, s->lv, bd, capL, 0, gcn, kPairCapG, scol_g, sfr_g, nullptr, dz + DZ_ROW_OVF, st,
                            nullptr, nld);
        launch_ds_check(dz, 6, 0u, dz + DZ_ROW_OVF, st);
        scan_exclusive_u32(hc, hrow, capL, dz + DZ_NPH, tmp, st);
        scan_exclusive_u32(gcn, grow, capL, dz + DZ_NPG, tmp, st);
        launch_ds_check(dz, 1, s->ds_cap_ph, nullptr, st);
        launch_ds_check(dz, 5, s->ds_cap_pg, nullptr, st);
        CK(cudaMemcpyAsync(hrow + capL, dz + DZ_NPH, sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(grow + capL, dz + DZ_NPG, sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
        launch_pair_compact(capL, kPairCapH, hc, hrow, scol_h, sfr_h, s->pscr_st.as<uint32_t>(),
                            s->hcol.as<uint32_t>(), s->hfr.as<float4>(), s->hsj.as<uint32_t>(), st, nld);
        launch_pair_compact(capL, kPairCapG, gcn, grow, scol_g, sfr_g, nullptr, s->gcol.as<uint32_t>(),
                            s->gfr.as<float4>(), nullptr, st, nld);
    } else {
        launch_pair_count(nd, s->lv, bd, capL, 1, hc, st, nullptr, nld);
        launch_pair_count(nd, s->lv, bd, capL, 0, gcn, st, nullptr, nld);
        scan_exclusive_u32(hc, hrow, capL, dz + DZ_NPH, tmp, st);
        scan_exclusive_u32(gcn, grow, capL, dz + DZ_NPG, tmp, st);
        launch_ds_check(dz, 1, s->ds_cap_ph, nullptr, st);
        launch_ds_check(dz, 5, s->ds_cap_pg, nullptr, st);
        CK(cudaMemcpyAsync(hrow + capL, dz + DZ_NPH, sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(grow + capL, dz + DZ_NPG, sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
        launch_pair_fill(nd, s->lv, bd, capL, 1, hrow, s->hcol.as<uint32_t>(), s->hfr.as<float4>(),
                         s->hsj.as<uint32_t>(), st, nullptr, nld);
        launch_pair_fill(nd, s->lv, bd, capL, 0, grow, s->gcol.as<uint32_t>(), s->gfr.as<float4>(), nullptr, st,
                         nullptr, nld);
    }
    uint32_t *gc = s->grp_cnt.as<uint32_t>(), *go = s->grp_off.as<uint32_t>();
    launch_group_count(s->lv, capL, 1, gc, st, nld);
    launch_group_count(s->lv, capL, 0, gc + nl, st, nld);
    scan_exclusive_u32(gc, go, capL, dz + DZ_GGAS, tmp, st);
    scan_exclusive_u32(gc + nl, go + nl, capL, dz + DZ_GALL, tmp, st);
    launch_ds_check(dz, 2, 0u, nullptr, st);
    launch_group_fill(s->lv, capL, 1, go, s->grp_gas.as<uint2>(), st, nld);
    launch_group_fill(s->lv, capL, 0, go + nl, s->grp_all.as<uint2>(), st, nld);
    // the passes over device work queues
    PassArgs a = pass_args(s);
    a.nleaf = capL;
    a.n_ggas = capI;
    a.n_gall = capI;
    a.ggas_dev = dz + DZ_GGAS;
    a.gall_dev = dz + DZ_GALL;
    a.queue = dz + DZ_QUEUE;
    a.nbr_count = nullptr;
    a.nbr_hash = nullptr;
    a.grav_count = nullptr;
    a.grav_hash = nullptr;
    a.nl_cnt = s->nl_cnt.as<uint32_t>();
    a.nl_len = s->nl_len.as<uint32_t>();
    a.nl_row = s->nl_row.as<uint32_t>();
    a.nl_j = s->nl_j.as<uint32_t>();
    a.nl_bound = 1;
    launch_records(a, mixed, st);
    // S3: lists (rows from the last step's counts) with the density in the fill
    CK(cudaMemsetAsync(a.nl_len, 0, (size_t)capI * sizeof(uint32_t), st));
    CK(cudaMemsetAsync(a.nl_retry, 0, sizeof(uint32_t), st));
    launch_hlist_bound(a, s->cnt_by_id.as<uint32_t>(), st);
    scan_exclusive_u32(a.nl_len, a.nl_row, capI, dz + DZ_ROWS, tmp, st);
    launch_ds_check(dz, 3, s->ds_cap_rows, nullptr, st);
    launch_hlist_fill(a, mixed, s->cap, false, st);
    launch_ds_check(dz, 4, 0u, a.nl_retry, st);
    launch_keep_counts(a, s->cnt_by_id.as<uint32_t>(), st);
    // S4-S8
    launch_moments(a, mixed, s->cap, st);
    launch_hydro(a, mixed, s->cap, st);
    launch_gravity(a, mixed, s->cap, false, st);
    launch_final_kick(a, mixed, s->nfloor.as<unsigned long long>(), st);
    return CRK_OK;
}

// Steps a handle can run as graph replays: the handle's own particles on a
// stream of its own, every leaf sorted every step, no mesh, no service pool.
static bool graph_eligible(const crk_sim *s)
{
    return !(s->prm.flags & CRK_FLAG_NO_GRAPH) && !s->timing && s->prm.pm_grid == 0 && !s->is_pool &&
           s->prm.rebuild_every <= 1 && s->n > 0 && s->n_dead == 0 && s->nleaf > 0;
}

// Capacities of the device-sized step from the last host-sized step, and
// every buffer it uses grown to them (before a capture: no allocation may
// happen inside one).
static int ds_prepare(crk_sim *s)
{
    const int64_t n = s->n;
    const double m = s->ds_margin;
    s->ds_cap_leaf = (int)std::min<int64_t>(n, (int64_t)(m * s->nleaf) + 64);
    s->ds_cap_items = (uint32_t)std::min<int64_t>((int64_t)4 * s->ds_cap_leaf, s->ds_cap_leaf + n / 32 + 64);
    s->ds_cap_rows = (uint32_t)((int64_t)(m * s->nl_rows) + 256);
    s->ds_cap_ph = (uint32_t)std::min<int64_t>((int64_t)(m * s->npair_h) + 256, 0xffffffffll);
    s->ds_cap_pg = (uint32_t)std::min<int64_t>((int64_t)(m * s->npair_g) + 256, 0xffffffffll);
    const size_t nl = (size_t)s->ds_cap_leaf, ni = s->ds_cap_items;
    const size_t cph = s->ds_cap_ph, cpg = s->ds_cap_pg;
    RET(s->dz.ensure(DZ_WORDS * sizeof(uint32_t)));
    RET(s->hcol.ensure(cph * 4));
    RET(s->hfr.ensure(cph * 16));
    RET(s->hsj.ensure(cph * 4));
    RET(s->gcol.ensure(cpg * 4));
    RET(s->gfr.ensure(cpg * 16));
    // the first step's walk fitted its fixed rows: walk once, as it did
    s->ds_one_walk = s->pair_two_pass_left == 0;
    if (s->ds_one_walk) {
        RET(s->pscr_col.ensure(nl * (kPairCapH + kPairCapG) * sizeof(uint32_t)));
        RET(s->pscr_fr.ensure(nl * (kPairCapH + kPairCapG) * sizeof(float4)));
        RET(s->pscr_st.ensure(nl * kPairCapH * sizeof(uint32_t)));
    }
    RET(s->grp_cnt.ensure(nl * 4 * 2));
    RET(s->grp_off.ensure(nl * 4 * 2));
    RET(s->grp_gas.ensure(ni * sizeof(uint2)));
    RET(s->grp_all.ensure(ni * sizeof(uint2)));
    RET(s->nl_cnt.ensure((size_t)std::max<int64_t>(n, 1) * 4));
    RET(s->nl_len.ensure(ni * 4));
    RET(s->nl_row.ensure(ni * 4));
    RET(s->nl_j.ensure((size_t)s->ds_cap_rows * 32u * 4u));
    const size_t words = (size_t)n;
    RET(s->ds_snap.ensure(words * (13 * sizeof(double) + 1 + 4 + 4 + 1)));
    if (!s->cap_st) CK(cudaStreamCreateWithFlags(&s->cap_st, cudaStreamNonBlocking));
    return CRK_OK;
}

// Two device-sized steps captured into the handle's graph (the state buffers
// swap at each sort, so two steps bring them back).  The capture runs on a
// stream of the library's own, so that handles on the legacy default stream
// can replay graphs too.
static int ds_capture(crk_sim *s)
{
    if (s->graph) {
        cudaGraphExecDestroy(s->graph);
        s->graph = nullptr;
    }
    cudaStream_t user = s->st;
    s->st = s->cap_st;
    const int64_t l0 = launches_so_far();
    cudaError_t e = cudaStreamBeginCapture(s->st, cudaStreamCaptureModeRelaxed);
    int rc = e == cudaSuccess ? CRK_OK : fail(CRK_ECUDA, "stream capture failed: %s", cudaGetErrorString(e));
    if (rc == CRK_OK) rc = run_step_ds(s);
    if (rc == CRK_OK) rc = run_step_ds(s);
    cudaGraph_t g = nullptr;
    if (e == cudaSuccess) {
        cudaError_t e2 = cudaStreamEndCapture(s->st, &g);
        if (rc == CRK_OK && e2 != cudaSuccess)
            rc = fail(CRK_ECUDA, "stream capture failed: %s", cudaGetErrorString(e2));
    }
    s->st = user;
    if (rc == CRK_OK) {
        e = cudaGraphInstantiate(&s->graph, g, 0);
        if (e != cudaSuccess) {
            s->graph = nullptr;
            rc = fail(CRK_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
        }
    }
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    s->graph_launch_nodes = (launches_so_far() - l0) / 2;
    return rc;
}

// Copies the state arrays (sorted order) to or from the batch snapshot.
static int ds_snapshot(crk_sim *s, bool save)
{
    const size_t n = (size_t)s->n;
    char *p = s->ds_snap.as<char>();
    double *dp[13] = {s->sa.x, s->sa.y, s->sa.z, s->sa.vx, s->sa.vy, s->sa.vz, s->sa.u, s->sa.m, s->sa.h,
                      s->sa.ax, s->sa.ay, s->sa.az, s->sa.du};
    auto cp = [&](void *dev, size_t bytes) -> int {
        CK(cudaMemcpyAsync(save ? (void *)p : dev, save ? dev : (void *)p, bytes, cudaMemcpyDeviceToDevice, s->st));
        p += bytes;
        return CRK_OK;
    };
    for (double *d : dp) RET(cp(d, n * sizeof(double)));
    RET(cp(s->sa.species, n));
    RET(cp(s->sa.slot, n * 4));
    RET(cp(s->sa.id, n * 4));
    RET(cp(s->sa.bin, n));
    return CRK_OK;
}

// nsteps KDK steps after the first ones: pairs of steps replayed from the
// captured graph, with one host synchronisation per call to read the
// overflow bits and the error word.  After an overflow the state of the
// batch start is restored, the capacities grow and the steps run host-sized.
static int step_graph(crk_sim *s, const double *dt, int nsteps)
{
    const int pairs = nsteps / 2;
    // the step sizes every replay uses live in the device box table
    for (int b = 0; b < s->nbox; ++b) {
        s->boxes[b].dt = dt[b];
        s->boxes[b].hdt = 0.5 * dt[b];
    }
    RET(upload_boxes(s));
    RET(ds_prepare(s));
    RET(ds_capture(s));
    RET(reset_error(s));
    RET(ds_snapshot(s, true));
    CK(cudaMemsetAsync(s->dz.p, 0, DZ_WORDS * sizeof(uint32_t), s->st));
    for (int k = 0; k < pairs; ++k) CK(cudaGraphLaunch(s->graph, s->st));
    note_launches((int)(2 * pairs * s->graph_launch_nodes));
    uint32_t ovf = 0;
    CK(cudaMemcpyAsync(s->host_scalars + 15, s->dz.as<uint32_t>() + DZ_OVF, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                       s->st));
    RET(read_error(s));
    ovf = s->host_scalars[15];
    s->tree_valid = false;  // the host's leaf and list sizes are those of the last host-sized step
    if (ovf == 0) {
        s->graph_steps += 2 * pairs;
        s->steps_run += 2 * pairs;
    } else {
        ++s->graph_overflows;
        s->ds_margin *= 1.5;
        RET(ds_snapshot(s, false));
        for (int k = 0; k < 2 * pairs; ++k) RET(run_step(s, dt, false));
    }
    for (int k = 2 * pairs; k < nsteps; ++k) RET(run_step(s, dt, false));
    return CRK_OK;
}

extern "C" int crk_step_boxes(crk_sim *s, const double *dt, int nsteps)
{
    if (!s || !dt) return fail(CRK_EINVAL, "null argument");
    if (nsteps < 0) return fail(CRK_EINVAL, "nsteps must be >= 0");
    for (int b = 0; b < s->nbox; ++b)
        if (!(dt[b] >= 0.0) || !std::isfinite(dt[b])) return fail(CRK_EINVAL, "dt must be finite and >= 0");
    CK(cudaSetDevice(s->device));
    if (s->n == 0) return CRK_OK;
    if (!s->have_forces) RET(run_step(s, nullptr, false));
    // the first step host-sized (it sizes the capacities), the rest replayed
    if (nsteps >= 3 && graph_eligible(s)) {
        RET(run_step(s, dt, false));
        if (graph_eligible(s)) return step_graph(s, dt, nsteps - 1);
        nsteps -= 1;
    }
    for (int k = 0; k < nsteps; ++k) RET(run_step(s, dt, false));
    return CRK_OK;
}

// One substep of the hierarchical steps (paper Sec. II and IV-B1): opening
// kicks and the drift, leaves sorted at the start of the long step and kept
// (boxes grown) in its other substeps, then the passes over the active part
// only: forces (hydro, gravity) for the leaves holding a particle whose step
// ends now, corrections for those and their hydro neighbour leaves, density
// and lists one ring of leaves further out; closing kicks and new bins.
static int run_substep(crk_sim *s, int sub, int depth, double dt_long, double eta, double courant,
                       unsigned long long *nactive)
{
    cudaStream_t st = s->st;
    const double d = std::ldexp(dt_long, -depth);
    RET(reset_error(s));
    if (s->timing) cudaEventRecord(s->ev_all[0], st);
    for (bool &r : s->recorded) r = false;
    const int64_t launches0 = launches_so_far();
    mark(s, PH_KICK, 0);
    launch_kick_drift_bins(s->sa, s->boxes_d.as<BoxDev>(), s->n, sub, depth, d,
                           s->nfloor.as<unsigned long long>(), st);
    mark(s, PH_KICK, 1);
    // particles active at t_(sub+1): bin >= depth - trailing_zeros(sub + 1);
    // the tree build flags their leaves (fh) and gives only those gravity rows
    const int t = sub + 1;
    int tz = 0;
    while (!((t >> tz) & 1)) ++tz;
    const int bmin = depth - tz;
    s->bins_bmin = bmin;
    const int rc_tree = build_tree(s, sub == 0 ? TREE_SORT : TREE_KEEP);
    s->bins_bmin = -1;
    RET(rc_tree);
    const size_t nl = (size_t)std::max(s->nleaf, 1);
    uint8_t *fh = s->bflag.as<uint8_t>(), *fm = fh + nl, *fd = fm + nl;
    launch_leaf_expand(s->hrow.as<uint32_t>(), s->hcol.as<uint32_t>(), s->nleaf, fh, fm, st);
    launch_leaf_expand(s->hrow.as<uint32_t>(), s->hcol.as<uint32_t>(), s->nleaf, fm, fd, st);
    const size_t ng = (size_t)std::max<uint32_t>(std::max(s->n_ggas, s->n_gall), 1);
    for (int k = 0; k < 4; ++k) RET(s->bgrp[k].ensure(ng * sizeof(uint2)));
    for (int k = 0; k < 2; ++k) RET(s->bmap[k].ensure(ng * sizeof(uint32_t)));
    RET(s->bkeep.ensure(ng * sizeof(uint32_t)));
    RET(s->bpos.ensure(ng * sizeof(uint32_t)));
    uint32_t *sc = s->scalars.as<uint32_t>(), *tmp = s->scan_tmp.as<uint32_t>();
    uint32_t *keep = s->bkeep.as<uint32_t>(), *pos = s->bpos.as<uint32_t>();
    uint2 *gD = s->bgrp[0].as<uint2>(), *gM = s->bgrp[1].as<uint2>(), *gH = s->bgrp[2].as<uint2>(),
          *gG = s->bgrp[3].as<uint2>();
    // gM: lists and density (the moments groups); gD: the outer ring, density
    // alone; gG: gravity
    launch_group_select(s->grp_gas.as<uint2>(), s->n_ggas, fm, keep, pos, sc + 9, tmp, gM, nullptr, st);
    launch_group_select(s->grp_gas.as<uint2>(), s->n_ggas, fd, keep, pos, sc + 8, tmp, gD, nullptr, st, fm);
    launch_group_select(s->grp_all.as<uint2>(), s->n_gall, fh, keep, pos, sc + 11, tmp, gG, nullptr, st);
    CK(cudaMemcpyAsync(s->host_scalars + 8, sc + 8, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(s->host_scalars + 11, sc + 11, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    HOST_SYNC(s);
    const uint32_t nD = s->host_scalars[8], nM = s->host_scalars[9], nG = s->host_scalars[11];
    // the hydro groups are taken from the moments groups, so that each keeps
    // the list row the fill pass wrote for it
    launch_group_select(gM, nM, fh, keep, pos, sc + 10, tmp, gH, s->bmap[1].as<uint32_t>(), st);
    CK(cudaMemcpyAsync(s->host_scalars + 10, sc + 10, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    HOST_SYNC(s);
    const uint32_t nH = s->host_scalars[10];

    PassArgs a = pass_args(s);
    a.nbr_count = nullptr;
    a.nbr_hash = nullptr;
    a.grav_count = nullptr;
    a.grav_hash = nullptr;
    // gravity rows exist only for the active leaves and hydro runs over the
    // active groups only: a pair must be seen from its own target's side, so
    // the gather forms
    a.grav_once = 0;
    a.hydro_once = 0;
    a.bsub = sub;
    a.bdepth = depth;
    a.bd = d;
    const int mixed = s->mixed ? 1 : 0;
    PassArgs aM = a, aD = a, aG = a;
    aM.ggas = gM;
    aM.n_ggas = nM;
    aD.ggas = gD;
    aD.n_ggas = nD;
    aG.gall = gG;
    aG.n_gall = nG;
    mark(s, PH_D, 0);
    launch_records(a, mixed, st);
    RET(density_pass(s, aM, false));
    launch_density_only(aD, mixed, s->cap, st);
    PassArgs aH = aM;
    aH.ggas = gH;
    aH.n_ggas = nH;
    aH.lmap = s->bmap[1].as<uint32_t>();
    mark(s, PH_D, 1);
    mark(s, PH_M, 0);
    launch_moments(aM, mixed, s->cap, st);
    mark(s, PH_M, 1);
    mark(s, PH_H, 0);
    launch_hydro(aH, mixed, s->cap, st);
    mark(s, PH_H, 1);
    mark(s, PH_G, 0);
    launch_gravity(aG, mixed, s->cap, false, st);
    mark(s, PH_G, 1);
    mark(s, PH_KDK, 0);
    launch_close_bins(a, mixed, sub, depth, d, dt_long, eta, courant, bmin, s->nfloor.as<unsigned long long>(),
                      nactive, st);
    mark(s, PH_KDK, 1);
    if (s->timing) cudaEventRecord(s->ev_all[1], st);
    CK(cudaGetLastError());
    RET(read_error(s));
    if (s->timing) {
        for (int ph = 0; ph < PH_N; ++ph) {
            if (!s->recorded[ph]) continue;
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, s->ev[ph][0], s->ev[ph][1]) == cudaSuccess) s->acc_ms[ph] += ms;
            else cudaGetLastError();
        }
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, s->ev_all[0], s->ev_all[1]) == cudaSuccess) s->total_ms += ms;
        else cudaGetLastError();
        s->calls++;
        s->launches += launches_so_far() - launches0;
    }
    return CRK_OK;
}

extern "C" int crk_step_bins(crk_sim *s, double dt_long, int depth, int nlong, double eta, double courant,
                             int64_t *active_counts)
{
    if (!s) return fail(CRK_EINVAL, "null handle");
    if (!(dt_long > 0.0) || !std::isfinite(dt_long)) return fail(CRK_EINVAL, "dt_long must be finite and > 0");
    if (depth < 0 || depth > 20) return fail(CRK_EINVAL, "depth in [0, 20]");
    if (nlong < 0) return fail(CRK_EINVAL, "nlong must be >= 0");
    if (!(eta > 0.0) || !(courant > 0.0) || !std::isfinite(eta) || !std::isfinite(courant))
        return fail(CRK_EINVAL, "eta and courant must be finite and > 0");
    CK(cudaSetDevice(s->device));
    const int nsub = 1 << depth;
    const size_t ncount = (size_t)nlong * (size_t)nsub;
    if (s->n == 0) {
        if (active_counts)
            for (size_t k = 0; k < ncount; ++k) active_counts[k] = 0;
        return CRK_OK;
    }
    // With a mesh the long-range force kicks on the long step (two half kicks
    // around it, the mesh at the positions of its start and its end) and the
    // substeps, their stored rates and the bins see the short-range and hydro
    // forces alone, so those are evaluated afresh first.
    const bool mesh = s->prm.pm_grid > 0;
    s->pm_suspend = mesh;
    int rc = CRK_OK;
    if (mesh || !s->have_forces) rc = run_step(s, nullptr, false);
    if (rc == CRK_OK) rc = s->bcount.ensure(std::max<size_t>(ncount, 1) * sizeof(unsigned long long));
    unsigned long long *cnt = s->bcount.as<unsigned long long>();
    if (rc == CRK_OK) {
        // every particle starts the long step with the bin of its stored rates
        launch_assign_bins(s->sa, s->boxes_d.as<BoxDev>(), s->n, dt_long, depth, eta, courant, s->st);
        if (cudaMemsetAsync(cnt, 0, std::max<size_t>(ncount, 1) * sizeof(unsigned long long), s->st) != cudaSuccess)
            rc = fail(CRK_ECUDA, "cudaMemsetAsync failed");
    }
    auto mesh_kick = [&]() {
        int r = pm_accelerations(s, s->acc_pm.as<double>(), false);
        if (r == CRK_OK) launch_pm_kick(s->sa, s->acc_pm.as<double>(), s->n, 0.5 * dt_long, s->st);
        return r;
    };
    for (int L = 0; L < nlong && rc == CRK_OK; ++L) {
        if (mesh) rc = mesh_kick();
        for (int sub = 0; sub < nsub && rc == CRK_OK; ++sub)
            rc = run_substep(s, sub, depth, dt_long, eta, courant, cnt + (size_t)L * nsub + sub);
        if (mesh && rc == CRK_OK) rc = mesh_kick();
    }
    s->pm_suspend = false;
    // the stored rates are the short-range part alone: a later fixed step
    // evaluates the full forces first
    if (mesh) s->have_forces = false;
    RET(rc);
    if (active_counts && ncount > 0) {
        std::vector<unsigned long long> h(ncount);
        CK(cudaMemcpyAsync(h.data(), cnt, ncount * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s->st));
        CK(cudaStreamSynchronize(s->st));
        for (size_t k = 0; k < ncount; ++k) active_counts[k] = (int64_t)h[k];
    }
    return CRK_OK;
}

extern "C" int crk_get_bins(crk_sim *s, uint8_t *bins, int mem)
{
    if (!s || (!bins && s->n > 0)) return fail(CRK_EINVAL, "null argument");
    if (mem != CRK_MEM_HOST && mem != CRK_MEM_DEVICE) return fail(CRK_EINVAL, "bad mem flag");
    CK(cudaSetDevice(s->device));
    const size_t n = (size_t)s->n;
    if (n == 0) return CRK_OK;
    if (mem == CRK_MEM_DEVICE) {
        launch_unpermute_bins(s->sa, s->n, bins, s->st);
    } else {
        RET(s->staging.ensure(n));
        launch_unpermute_bins(s->sa, s->n, s->staging.as<uint8_t>(), s->st);
        CK(cudaMemcpyAsync(bins, s->staging.p, n, cudaMemcpyDeviceToHost, s->st));
    }
    CK(cudaStreamSynchronize(s->st));
    return CRK_OK;
}

extern "C" int crk_step(crk_sim *s, double dt, int nsteps)
{
    if (!s) return fail(CRK_EINVAL, "null handle");
    std::vector<double> d((size_t)std::max(s->nbox, 1), dt);
    return crk_step_boxes(s, d.data(), nsteps);
}

extern "C" int crk_get_state(crk_sim *s, double *pos, double *vel, double *u, int mem)
{
    if (!s) return fail(CRK_EINVAL, "null handle");
    if (mem != CRK_MEM_HOST && mem != CRK_MEM_DEVICE) return fail(CRK_EINVAL, "bad mem flag");
    CK(cudaSetDevice(s->device));
    const size_t n = (size_t)s->n;
    if (n == 0) return CRK_OK;
    if (mem == CRK_MEM_DEVICE) {
        launch_unpermute_state(s->sa, s->n, pos, vel, u, s->st);
    } else {
        RET(s->staging.ensure(n * 8 * 7 + 1024));
        double *dp = s->staging.as<double>(), *dv = dp + 3 * n, *du = dv + 3 * n;
        launch_unpermute_state(s->sa, s->n, pos ? dp : nullptr, vel ? dv : nullptr, u ? du : nullptr, s->st);
        if (pos) CK(cudaMemcpyAsync(pos, dp, 3 * n * 8, cudaMemcpyDeviceToHost, s->st));
        if (vel) CK(cudaMemcpyAsync(vel, dv, 3 * n * 8, cudaMemcpyDeviceToHost, s->st));
        if (u) CK(cudaMemcpyAsync(u, du, n * 8, cudaMemcpyDeviceToHost, s->st));
    }
    CK(cudaStreamSynchronize(s->st));
    return CRK_OK;
}

extern "C" int crk_get_sums(crk_sim *s, double momentum[3], double *energy, int64_t *nfloor)
{
    if (!s) return fail(CRK_EINVAL, "null handle");
    CK(cudaSetDevice(s->device));
    double v[4] = {0, 0, 0, 0};
    unsigned long long nf = 0;
    if (s->n > 0) {
        launch_state_sums(s->sa, s->n, s->partial.as<double>(), sums_blocks(s->n), s->sums.as<double>(), s->st);
        CK(cudaMemcpyAsync(v, s->sums.p, sizeof v, cudaMemcpyDeviceToHost, s->st));
        CK(cudaMemcpyAsync(&nf, s->nfloor.p, 8, cudaMemcpyDeviceToHost, s->st));
        CK(cudaStreamSynchronize(s->st));
    }
    if (momentum) {
        momentum[0] = v[0];
        momentum[1] = v[1];
        momentum[2] = v[2];
    }
    if (energy) *energy = v[3];
    if (nfloor) *nfloor = (int64_t)nf;
    return CRK_OK;
}

extern "C" int crk_get_size(crk_sim *s, int64_t *n, int *nbox)
{
    if (!s) return fail(CRK_EINVAL, "null handle");
    if (n) *n = s->n;
    if (nbox) *nbox = s->nbox;
    return CRK_OK;
}

extern "C" int crk_set_timing(crk_sim *s, int enable)
{
    if (!s) return fail(CRK_EINVAL, "null handle");
    s->timing = enable != 0;
    for (double &v : s->acc_ms) v = 0;
    s->total_ms = 0;
    s->calls = 0;
    s->launches = 0;
    s->host_syncs = s->steps_run = s->graph_steps = s->graph_overflows = 0;
    return CRK_OK;
}

extern "C" int crk_fof(crk_sim *s, double b, int species_mask, int64_t *group, int64_t *ngroups, int mem)
{
    if (!s || !group || !ngroups) return fail(CRK_EINVAL, "null argument");
    if (species_mask < 1 || species_mask > 3) return fail(CRK_EINVAL, "species_mask must be 1, 2 or 3");
    if (mem != CRK_MEM_HOST && mem != CRK_MEM_DEVICE) return fail(CRK_EINVAL, "bad mem flag");
    if (!(b > 0.0)) return fail(CRK_EINVAL, "linking length must be > 0");
    for (const BoxDev &bx : s->boxes)
        if (bx.active && !(b <= bx.r_cut)) return fail(CRK_EINVAL, "linking length %g above r_cut %g", b, bx.r_cut);
    CK(cudaSetDevice(s->device));
    *ngroups = 0;
    if (s->n == 0) return CRK_OK;
    RET(reset_error(s));
    RET(build_tree(s));
    const size_t n = (size_t)s->n;
    RET(s->fof_par.ensure(n * 4 + 8 * 8));
    uint32_t *par = s->fof_par.as<uint32_t>();
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(par + ((n + 1) & ~size_t(1)));
    int64_t *dst = group;
    if (mem == CRK_MEM_HOST) {
        RET(s->staging.ensure(n * 8 + 256));
        dst = s->staging.as<int64_t>();
    }
    CK(cudaMemsetAsync(cnt, 0, 8, s->st));
    PassArgs a = pass_args(s);
    launch_fof(a, s->mixed ? 1 : 0, s->cap, par, b, species_mask, dst, cnt, s->st);
    CK(cudaGetLastError());
    unsigned long long h_cnt = 0;
    CK(cudaMemcpyAsync(&h_cnt, cnt, 8, cudaMemcpyDeviceToHost, s->st));
    if (mem == CRK_MEM_HOST) CK(cudaMemcpyAsync(group, dst, n * 8, cudaMemcpyDeviceToHost, s->st));
    RET(read_error(s));  // synchronises
    *ngroups = (int64_t)h_cnt;
    return CRK_OK;
}

extern "C" int crk_pm_accel(crk_sim *s, double *acc, int mem)
{
    if (!s || !acc) return fail(CRK_EINVAL, "null argument");
    if (mem != CRK_MEM_HOST && mem != CRK_MEM_DEVICE) return fail(CRK_EINVAL, "bad mem flag");
    if (s->prm.pm_grid <= 0) return fail(CRK_EINVAL, "the handle has no mesh (pm_grid = 0)");
    if (s->nbox != 1) return fail(CRK_EINVAL, "no box loaded");
    CK(cudaSetDevice(s->device));
    const size_t n = (size_t)s->n;
    double *dst = acc;
    if (mem == CRK_MEM_HOST) {
        RET(s->staging.ensure(std::max<size_t>(n, 1) * 3 * sizeof(double)));
        dst = s->staging.as<double>();
    }
    RET(pm_accelerations(s, dst, true));
    if (mem == CRK_MEM_HOST && n > 0)
        CK(cudaMemcpyAsync(acc, dst, n * 3 * sizeof(double), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    return CRK_OK;
}

// Times one force evaluation (after a warm-up one) at every (capacity,
// gravity form) candidate and keeps the fastest.
static int autotune_grid(crk_sim *s, const int *caps, int ncaps, const int *forms, int nforms, int *best_cap,
                         int *best_form, double *ms_out)
{
    if (!s || !caps || ncaps < 1 || !forms || nforms < 1) return fail(CRK_EINVAL, "null argument or no candidate");
    for (int k = 0; k < ncaps; ++k)
        if (caps[k] != 32 && caps[k] != 64 && caps[k] != 128)
            return fail(CRK_EINVAL, "leaf capacity candidates must be 32, 64 or 128 (got %d)", caps[k]);
    for (int f = 0; f < nforms; ++f)
        if (forms[f] < 0 || forms[f] > (CRK_GRAVITY_PAIRS_ONCE | CRK_HYDRO_PAIRS_ONCE))
            return fail(CRK_EINVAL, "pair-decomposition candidates are bit sets of CRK_GRAVITY_PAIRS_ONCE "
                                    "and CRK_HYDRO_PAIRS_ONCE (got %d)", forms[f]);
    CK(cudaSetDevice(s->device));
    if (s->n == 0) return fail(CRK_EINVAL, "no particles loaded");
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(CRK_ECUDA, "event creation failed: %s", cudaGetErrorString(ce));
    }
    const int once_bits = CRK_FLAG_GRAVITY_PAIRS_ONCE | CRK_FLAG_HYDRO_PAIRS_ONCE;
    const int flags0 = s->prm.flags & ~once_bits;
    auto flags_of = [&](int form) {
        return flags0 | ((form & CRK_GRAVITY_PAIRS_ONCE) ? CRK_FLAG_GRAVITY_PAIRS_ONCE : 0) |
               ((form & CRK_HYDRO_PAIRS_ONCE) ? CRK_FLAG_HYDRO_PAIRS_ONCE : 0);
    };
    int best = -1;
    double best_ms = 0.0;
    int rc = CRK_OK;
    for (int k = 0; k < ncaps && rc == CRK_OK; ++k) {
        s->cap = caps[k];
        s->tree_valid = false;  // leaves of another capacity
        for (int f = 0; f < nforms && rc == CRK_OK; ++f) {
            s->prm.flags = flags_of(forms[f]);
            rc = run_step(s, nullptr, false);  // warm-up: buffers grow to this layout
            if (rc != CRK_OK) break;
            cudaEventRecord(e0, s->st);
            rc = run_step(s, nullptr, false);
            cudaEventRecord(e1, s->st);
            if (rc != CRK_OK) break;
            float ms = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                rc = fail(CRK_ECUDA, "event timing failed");
                break;
            }
            if (ms_out) ms_out[k * nforms + f] = ms;
            if (best < 0 || ms < best_ms) {
                best = k * nforms + f;
                best_ms = ms;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != CRK_OK) return rc;
    const int bc = caps[best / nforms], bf = forms[best % nforms];
    s->cap = bc;
    s->prm.flags = flags_of(bf);
    s->tree_valid = false;
    if (best_cap) *best_cap = bc;
    if (best_form) *best_form = bf;
    // the stored accelerations are those of the chosen configuration
    return run_step(s, nullptr, false);
}

extern "C" int crk_autotune(crk_sim *s, const int *caps, int ncaps, int *best_cap, double *ms_out)
{
    if (!s) return fail(CRK_EINVAL, "null handle");
    const int form = ((s->prm.flags & CRK_FLAG_GRAVITY_PAIRS_ONCE) ? CRK_GRAVITY_PAIRS_ONCE : 0) |
                     ((s->prm.flags & CRK_FLAG_HYDRO_PAIRS_ONCE) ? CRK_HYDRO_PAIRS_ONCE : 0);
    return autotune_grid(s, caps, ncaps, &form, 1, best_cap, nullptr, ms_out);
}

extern "C" int crk_autotune_ex(crk_sim *s, const int *caps, int ncaps, const int *forms, int nforms, int *best_cap,
                               int *best_form, double *ms_out)
{
    return autotune_grid(s, caps, ncaps, forms, nforms, best_cap, best_form, ms_out);
}

extern "C" int crk_set_state(crk_sim *s, const double *pos, const double *vel, const double *u,
                             int mem)
{
    if (!s) return fail(CRK_EINVAL, "null handle");
    if (mem != CRK_MEM_HOST && mem != CRK_MEM_DEVICE) return fail(CRK_EINVAL, "bad mem flag");
    CK(cudaSetDevice(s->device));
    const size_t n = (size_t)s->n;
    if (n == 0) return CRK_OK;
    const double *dp = pos, *dv = vel, *du = u;
    if (mem == CRK_MEM_HOST) {
        RET(s->in_stage.ensure(n * 7 * 8 + 64));
        double *b = s->in_stage.as<double>();
        if (pos) CK(cudaMemcpyAsync(b, pos, n * 24, cudaMemcpyHostToDevice, s->st));
        if (vel) CK(cudaMemcpyAsync(b + 3 * n, vel, n * 24, cudaMemcpyHostToDevice, s->st));
        if (u) CK(cudaMemcpyAsync(b + 6 * n, u, n * 8, cudaMemcpyHostToDevice, s->st));
        dp = pos ? b : nullptr;
        dv = vel ? b + 3 * n : nullptr;
        du = u ? b + 6 * n : nullptr;
    }
    launch_set_state(s->sa, s->n, dp, dv, du, s->st);
    RET(reset_error(s));
    launch_validate(s->sa, s->boxes_d.as<BoxDev>(), s->n, s->err.as<int>(), s->st);
    CK(cudaGetLastError());
    return read_error(s);
}

extern "C" int crk_get_timings(crk_sim *s, crk_timings *t)
{
    if (!s || !t) return fail(CRK_EINVAL, "null argument");
    t->tree_ms = s->acc_ms[PH_TREE];
    t->pairs_ms = s->acc_ms[PH_PAIRS];
    t->density_ms = s->acc_ms[PH_D];
    t->moments_ms = s->acc_ms[PH_M];
    t->hydro_ms = s->acc_ms[PH_H];
    t->gravity_ms = s->acc_ms[PH_G];
    t->kdk_ms = s->acc_ms[PH_KDK] + s->acc_ms[PH_KICK];
    t->total_ms = s->total_ms;
    t->calls = s->calls;
    t->pairs_hydro = s->npair_h;
    t->pairs_grav = s->npair_g;
    t->nleaves = s->nleaf;
    t->launches = s->launches;
    t->pm_ms = s->acc_ms[PH_PM];
    t->tests_hydro = (int64_t)s->census_h[0];
    t->list_entries = (int64_t)s->census_h[1];
    t->tests_grav = (int64_t)s->census_h[2];
    t->tests_grav_target = (int64_t)s->census_h[3];
    t->list_slots = 32 * s->census_rows;
    t->steps = s->steps_run;
    t->graph_steps = s->graph_steps;
    t->host_syncs = s->host_syncs;
    t->graph_overflows = s->graph_overflows;
    return CRK_OK;
}

extern "C" int crk_get_tree(crk_sim *s, crk_tree *t)
{
    if (!s || !t) return fail(CRK_EINVAL, "null argument");
    if (!s->tree_valid || (s->n > 0 && s->nleaf == 0))
        return fail(CRK_EINVAL, "no tree: call crk_forces or crk_step first");
    t->n = s->n;
    t->nleaf = s->nleaf;
    t->npair_hydro = s->npair_h;
    t->npair_grav = s->npair_g;
    const size_t nl = (size_t)s->nleaf;
    if (nl == 0) return CRK_OK;
    CK(cudaStreamSynchronize(s->st));
    auto get = [&](void *dst, const void *src, size_t bytes) -> int {
        if (dst && bytes) CK(cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost));
        return CRK_OK;
    };
    if (t->order && s->n > 0) {
        std::vector<uint32_t> id((size_t)s->n);
        RET(get(id.data(), s->sa.id, id.size() * sizeof(uint32_t)));
        for (size_t k = 0; k < id.size(); ++k) t->order[k] = (int64_t)id[k];
    }
    RET(get(t->leaf_start, s->lv.start, nl * sizeof(uint32_t)));
    RET(get(t->leaf_count, s->lv.count, nl * sizeof(uint32_t)));
    RET(get(t->leaf_species, s->lv.species, nl));
    if (t->leaf_centre && nl) {
        std::vector<double> c(3 * nl);
        RET(get(c.data(), s->lv.cx, nl * sizeof(double)));
        RET(get(c.data() + nl, s->lv.cy, nl * sizeof(double)));
        RET(get(c.data() + 2 * nl, s->lv.cz, nl * sizeof(double)));
        for (size_t L = 0; L < nl; ++L)
            for (int a = 0; a < 3; ++a) t->leaf_centre[3 * L + a] = c[a * nl + L];
    }
    if (t->leaf_half && nl) {
        std::vector<float> e(3 * nl);
        RET(get(e.data(), s->lv.ex, nl * sizeof(float)));
        RET(get(e.data() + nl, s->lv.ey, nl * sizeof(float)));
        RET(get(e.data() + 2 * nl, s->lv.ez, nl * sizeof(float)));
        for (size_t L = 0; L < nl; ++L)
            for (int a = 0; a < 3; ++a) t->leaf_half[3 * L + a] = e[a * nl + L];
    }
    RET(get(t->hydro_row, s->hrow.p, (nl + 1) * sizeof(uint32_t)));
    RET(get(t->hydro_col, s->hcol.p, (size_t)s->npair_h * sizeof(uint32_t)));
    RET(get(t->grav_row, s->grow.p, (nl + 1) * sizeof(uint32_t)));
    RET(get(t->grav_col, s->gcol.p, (size_t)s->npair_g * sizeof(uint32_t)));
    return CRK_OK;
}

extern "C" int crk_destroy(crk_sim *s)
{
    if (!s) return CRK_OK;
    cudaSetDevice(s->device);
    cudaStreamSynchronize(s->st);
    for (int k = 0; k < 17; ++k) {
        s->stA[k].release();
        s->stB[k].release();
    }
    DBuf *bufs[] = {&s->boxes_d, &s->keys, &s->keys_alt, &s->vals, &s->vals_alt, &s->counts,
                    &s->scan_tmp, &s->flags, &s->flag_scan, &s->scalars, &s->lv_sp, &s->lv_h,
                    &s->nd_slot, &s->hrow, &s->grow, &s->hcnt, &s->gcnt, &s->hcol, &s->gcol,
                    &s->pm, &s->uhat, &s->acc_h, &s->acc_g, &s->nbrc, &s->nbrh, &s->gravc,
                    &s->gravh, &s->err, &s->nfloor, &s->partial, &s->sums, &s->staging,
                    &s->in_stage, &s->grp_cnt, &s->grp_off, &s->grp_gas, &s->grp_all, &s->hfr, &s->gfr,
                    &s->nl_j, &s->nl_row, &s->nl_len, &s->nl_cnt, &s->hsj, &s->fof_par, &s->acc_pm,
                    &s->bflag, &s->bgrp[0], &s->bgrp[1], &s->bgrp[2], &s->bgrp[3], &s->bmap[0],
                    &s->bmap[1], &s->bkeep, &s->bpos, &s->bcount, &s->cnt_by_id, &s->nl_retry, &s->census, &s->pscr_col, &s->pscr_fr, &s->pscr_st,
                    &s->dz, &s->ds_snap};
    for (DBuf *b : bufs) b->release();
    pm_release(s);
    for (int k = 0; k < 3; ++k) {
        s->lv_u32[k].release();
        s->lv_c[k].release();
        s->lv_e[k].release();
        if (k < 2) s->lv_chunk[k].release();
    }
    for (int k = 0; k < 7; ++k) {
        s->nd_f[k].release();
        s->hrec[k].release();
    }
    for (int ph = 0; ph < PH_N; ++ph)
        for (int w = 0; w < 2; ++w)
            if (s->ev[ph][w]) cudaEventDestroy(s->ev[ph][w]);
    if (s->ev_all[0]) cudaEventDestroy(s->ev_all[0]);
    if (s->ev_all[1]) cudaEventDestroy(s->ev_all[1]);
    if (s->graph) cudaGraphExecDestroy(s->graph);
    if (s->cap_st) cudaStreamDestroy(s->cap_st);
    if (s->host_scalars) cudaFreeHost(s->host_scalars);
    if (s->host_err) cudaFreeHost(s->host_err);
    delete s;
    return CRK_OK;
}

// ------------------------------------------------------------------ pool
// A handle used by the service: its boxes are `max_slots` fixed slots; jobs
// are appended into free slots between steps and leave by deactivating their
// slot (their particles then sort last and are dropped at the next step).
namespace crk {

size_t pool_bytes_per_particle(const crk_sim *s)
{
    const size_t r = s->mixed ? 4 : 8;
    // two state copies, sort buffers, leaves/hierarchy bound, records, counts
    return 2 * (13 * 8 + 9) + 2 * 12 + 8 + 128 + 4 * r * 10 + r + 24 + 64;
}

int pool_init(crk_sim *s, int max_slots)
{
    if (max_slots < 1) return fail(CRK_EINVAL, "max_slots must be >= 1");
    s->is_pool = true;
    s->cnt_valid = false;
    if (s->prm.pm_grid > 0) return fail(CRK_EINVAL, "the service takes no mesh (pm_grid must be 0)");
    CK(cudaSetDevice(s->device));
    int sb = 0;
    while ((1 << sb) < max_slots + 1) ++sb;
    s->slot_bits = sb;
    s->nbox = max_slots;
    crk_physics dummy{};
    dummy.box = 1.0;
    dummy.r_cut = 0.1;
    dummy.r_split = 0.1;
    dummy.gamma = 5.0 / 3.0;
    // slots 0 .. max_slots-1 take jobs; slot max_slots holds retired particles
    s->boxes.assign((size_t)max_slots + 1, box_dev(dummy));
    for (BoxDev &b : s->boxes) b.active = 0;
    s->n = 0;
    s->tree_valid = false;
    s->n_dead = 0;
    RET(reserve(s, 4096));
    RET(upload_boxes(s));
    CK(cudaMemsetAsync(s->nfloor.p, 0, 8, s->st));
    return CRK_OK;
}

static State shifted(const State &a, int64_t off)
{
    State b = a;
    b.x += off; b.y += off; b.z += off;
    b.vx += off; b.vy += off; b.vz += off;
    b.u += off; b.m += off; b.h += off;
    b.ax += off; b.ay += off; b.az += off; b.du += off;
    b.species += off; b.slot += off; b.id += off; b.bin += off;
    return b;
}

static int pool_grow(crk_sim *s, int64_t need)
{
    if (need <= s->cap_n) return CRK_OK;
    const int64_t cap = std::max<int64_t>(need, 2 * s->cap_n);
    const size_t keep = (size_t)s->n;
    for (int k = 0; k < 13; ++k) RET(s->stA[k].ensure_keep((size_t)cap * 8, keep * 8, s->st));
    RET(s->stA[13].ensure_keep((size_t)cap, keep, s->st));
    RET(s->stA[14].ensure_keep((size_t)cap * 4, keep * 4, s->st));
    RET(s->stA[15].ensure_keep((size_t)cap * 4, keep * 4, s->st));
    RET(s->stA[16].ensure_keep((size_t)cap, keep, s->st));
    return reserve(s, cap);
}

int pool_add(crk_sim *s, int slot, const crk_physics &phys, int64_t n, const double *pos,
             const double *vel, const double *mass, const double *u, const double *h,
             const uint8_t *species, const double *acc, const double *dudt)
{
    if (slot < 0 || slot >= s->nbox) return fail(CRK_EINVAL, "bad slot %d", slot);
    RET(check_physics(phys));
    if (n <= 0) return fail(CRK_EINVAL, "a job needs at least one particle");
    CK(cudaSetDevice(s->device));
    const int64_t n0 = s->n;
    RET(pool_grow(s, n0 + n));
    int64_t ng = 0;
    for (int64_t k = 0; k < n; ++k) ng += species[k] == CRK_GAS;
    const int lvl = std::min(auto_cm_level(std::max(ng, n - ng), s->cap), (63 - s->slot_bits) / 3);
    BoxDev b = box_dev(phys);
    b.cm_shift = 63 - s->slot_bits - 3 * lvl;
    b.active = 1;
    s->boxes[slot] = b;
    RET(upload_boxes(s));
    const size_t nn = (size_t)n;
    RET(s->in_stage.ensure(nn * 13 * sizeof(double) + nn * 5 + 64));
    double *d_pos = s->in_stage.as<double>();
    double *d_vel = d_pos + 3 * nn, *d_mass = d_vel + 3 * nn, *d_u = d_mass + nn, *d_h = d_u + nn;
    double *d_acc = d_h + nn, *d_du = d_acc + 3 * nn;
    uint32_t *d_slot = (uint32_t *)(d_du + nn);
    uint8_t *d_sp = (uint8_t *)(d_slot + nn);
    std::vector<uint32_t> slot_of(nn, (uint32_t)slot);
    CK(cudaMemcpyAsync(d_pos, pos, nn * 24, cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(d_vel, vel, nn * 24, cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(d_mass, mass, nn * 8, cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(d_u, u, nn * 8, cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(d_h, h, nn * 8, cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(d_sp, species, nn, cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(d_slot, slot_of.data(), nn * 4, cudaMemcpyHostToDevice, s->st));
    const State part = shifted(s->sa, n0);
    launch_load_state(part, n, d_pos, d_vel, d_mass, d_u, d_h, d_sp, d_slot, s->st);
    if (acc && dudt) {
        CK(cudaMemcpyAsync(d_acc, acc, nn * 24, cudaMemcpyHostToDevice, s->st));
        CK(cudaMemcpyAsync(d_du, dudt, nn * 8, cudaMemcpyHostToDevice, s->st));
        launch_set_forces(part, n, d_acc, d_du, s->st);
    }
    RET(reset_error(s));
    launch_validate(part, s->boxes_d.as<BoxDev>(), n, s->err.as<int>(), s->st);
    CK(cudaGetLastError());
    int rc = read_error(s);  // synchronises: the host arrays may be released after return
    if (rc != CRK_OK) {
        s->boxes[slot].active = 0;
        upload_boxes(s);
        return rc;
    }
    s->n = n0 + n;
    s->tree_valid = false;
    return CRK_OK;
}

int pool_extract(crk_sim *s, int slot, int64_t n, double *pos, double *vel, double *u)
{
    CK(cudaSetDevice(s->device));
    const size_t nn = (size_t)n;
    RET(s->staging.ensure(nn * 7 * 8 + 256));
    double *dp = s->staging.as<double>(), *dv = dp + 3 * nn, *du = dv + 3 * nn;
    launch_extract_slot(s->sa, s->n, (uint32_t)slot, n, dp, dv, du, nullptr, nullptr, s->st);
    if (pos) CK(cudaMemcpyAsync(pos, dp, nn * 24, cudaMemcpyDeviceToHost, s->st));
    if (vel) CK(cudaMemcpyAsync(vel, dv, nn * 24, cudaMemcpyDeviceToHost, s->st));
    if (u) CK(cudaMemcpyAsync(u, du, nn * 8, cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    return CRK_OK;
}

int pool_snapshot(crk_sim *s, int slot, int64_t n, double *dev)
{
    CK(cudaSetDevice(s->device));
    const size_t nn = (size_t)n;
    double *dp = dev, *dv = dp + 3 * nn, *du = dv + 3 * nn, *da = du + nn, *dd = da + 3 * nn;
    launch_extract_slot(s->sa, s->n, (uint32_t)slot, n, dp, dv, du, da, dd, s->st);
    CK(cudaGetLastError());
    return CRK_OK;
}

int pool_remove(crk_sim *s, int slot, int64_t n)
{
    CK(cudaSetDevice(s->device));
    launch_retire_slot(s->sa, s->n, (uint32_t)slot, (uint32_t)s->nbox, s->st);
    CK(cudaGetLastError());
    s->boxes[slot].active = 0;
    s->n_dead += n;
    return CRK_OK;
}

int pool_step(crk_sim *s, const double *dt_per_slot)
{
    CK(cudaSetDevice(s->device));
    if (s->n == 0) return CRK_OK;
    return run_step(s, dt_per_slot, false);
}

}  // namespace crk
