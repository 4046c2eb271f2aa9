// Continuous-batching service for many small-box force-and-KDK jobs (the
// shape of an emulator campaign).  Jobs are sorted by size into classes
// (lanes); each lane owns a pool handle whose box slots hold its resident
// jobs' particles and trees on the device, its own CUDA stream and its own
// host thread.  Every iteration a lane admits queued jobs of its class into
// free slots while the shared HBM budget allows, advances all its resident
// jobs by one KDK step in the same batched launches (a newly admitted job's
// first step is its initial force evaluation, dt = 0), and publishes the jobs
// whose steps are done.  The lanes run side by side on the device, so a small
// job's step never waits for the largest box in the service.  The paper's
// GPU-resident design (Sec. IV-A: data stays on the device for the whole PM
// step) applied across jobs instead of across substeps.
//
// Locking: one mutex guards the ticket table, the queues, the slots, the
// budget and every job field that crk_poll or crk_service_snapshot reads;
// a job's final state and status are written under it before `done` is set.
#include "sim.h"

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

using namespace crk;

namespace {

using clk = std::chrono::steady_clock;

// Size classes: a job of n particles goes to the first lane whose upper
// bound exceeds n; lane k < K-1 takes n < 8192 * 8^(k+1) (65,536, 524,288,
// ...: one class per factor 8, a factor 2 in the lattice side n^(1/3)).
constexpr int kDefaultClasses = 3;
constexpr int kMaxClasses = 8;

int64_t class_bound(int k) { return (int64_t)8192 << (3 * (k + 1)); }

struct Job {
    uint64_t ticket = 0;
    crk_physics phys{};
    int64_t n = 0;
    int lane = 0;
    std::vector<double> pos, vel, mass, u, h;
    std::vector<double> acc, du;  // forces to resume with (empty: a fresh job)
    std::vector<uint8_t> sp;
    double dt = 0.0;
    int nsteps = 0;
    int steps_done = 0;
    bool init_done = false;
    bool cancel = false;
    int slot = -1;
    size_t bytes = 0;
    int status = CRK_OK;
    std::string msg;
    bool done = false;
    clk::time_point t_submit, t_admit, t_done;
    // snapshot: device staging (11 n doubles, allocated at admission), pinned
    // host copy (allocated at submission), completion event
    crk::DBuf snap_dev;
    double *snap_host = nullptr;
    cudaEvent_t snap_ev = nullptr;
    bool snap_inflight = false;
    int snap_steps = -1;          // steps of the copy in flight or last completed
    int snap_valid = -1;          // steps of the last completed copy (-1: none)

    ~Job()
    {
        snap_dev.release();
        if (snap_host) cudaFreeHost(snap_host);
        if (snap_ev) cudaEventDestroy(snap_ev);
    }
};

struct Lane {
    int index = 0;
    crk_sim *sim = nullptr;
    cudaStream_t st = nullptr;
    cudaStream_t side = nullptr;  // snapshot copies
    cudaEvent_t stepped = nullptr;
    std::thread th;
    std::condition_variable cv_work;
    std::deque<std::shared_ptr<Job>> pending;
    std::vector<std::shared_ptr<Job>> slots;
};

}  // namespace

struct crk_service {
    crk_service_params prm{};
    size_t bpp = 0;
    std::mutex mu;
    std::condition_variable cv_done;
    std::vector<std::unique_ptr<Lane>> lanes;
    std::unordered_map<uint64_t, std::shared_ptr<Job>> jobs;
    uint64_t next_ticket = 1;
    size_t resident_bytes = 0;
    bool stop = false;
};

namespace {

// Marks a job finished.  Caller holds sv->mu.
void finish_locked(const std::shared_ptr<Job> &j, int status, const char *msg)
{
    j->status = status;
    if (msg) j->msg = msg;
    j->t_done = clk::now();
    j->done = true;
}

// Starts a snapshot of a resident job: extraction on the lane's stream,
// device-to-host copy on its side stream (overlapping the next step).  The
// previous copy of the job is completed first (its staging is reused).
// Both buffers exist already.  Caller holds sv->mu.
int start_snapshot(Lane &ln, Job &j)
{
    const size_t words = (size_t)j.n * 11;
    if (j.snap_inflight) {
        CK(cudaEventSynchronize(j.snap_ev));
        j.snap_valid = j.snap_steps;
        j.snap_inflight = false;
    }
    RET(pool_snapshot(ln.sim, j.slot, j.n, j.snap_dev.as<double>()));
    CK(cudaEventRecord(ln.stepped, ln.st));
    CK(cudaStreamWaitEvent(ln.side, ln.stepped, 0));
    CK(cudaMemcpyAsync(j.snap_host, j.snap_dev.p, words * sizeof(double), cudaMemcpyDeviceToHost, ln.side));
    CK(cudaEventRecord(j.snap_ev, ln.side));
    j.snap_steps = j.steps_done;
    j.snap_inflight = true;
    return CRK_OK;
}

// Final state of a job, copied out of its slot without the lock, then
// published under it.
struct Extracted {
    std::vector<double> pos, vel, u;
    int rc = CRK_OK;
    std::string msg;
};

Extracted extract(Lane &ln, const Job &j)
{
    Extracted e;
    e.pos.resize((size_t)j.n * 3);
    e.vel.resize((size_t)j.n * 3);
    e.u.resize((size_t)j.n);
    e.rc = pool_extract(ln.sim, j.slot, j.n, e.pos.data(), e.vel.data(), e.u.data());
    if (e.rc != CRK_OK) e.msg = crk_last_error();
    return e;
}

void publish_locked(const std::shared_ptr<Job> &j, Extracted &e)
{
    if (e.rc == CRK_OK) {
        j->pos.swap(e.pos);
        j->vel.swap(e.vel);
        j->u.swap(e.u);
    }
    finish_locked(j, e.rc, e.rc == CRK_OK ? nullptr : e.msg.c_str());
}

void worker(crk_service *sv, Lane *ln)
{
    cudaSetDevice(sv->prm.device);
    std::vector<double> dts((size_t)sv->prm.max_slots, 0.0);
    while (true) {
        std::vector<std::shared_ptr<Job>> admitted;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            // FIFO admission of this class while a slot and the budget allow.
            while (!ln->pending.empty()) {
                auto &j = ln->pending.front();
                int free_slot = -1;
                for (int s = 0; s < sv->prm.max_slots; ++s)
                    if (!ln->slots[s]) {
                        free_slot = s;
                        break;
                    }
                if (free_slot < 0 || sv->resident_bytes + j->bytes > sv->prm.hbm_budget_bytes) break;
                j->slot = free_slot;
                ln->slots[free_slot] = j;
                sv->resident_bytes += j->bytes;
                admitted.push_back(j);
                ln->pending.pop_front();
            }
            bool any = false;
            for (auto &p : ln->slots) any = any || (p != nullptr);
            if (!any) {
                if (sv->stop) break;
                ln->cv_work.wait(lk);
                continue;
            }
        }
        std::vector<std::shared_ptr<Job>> leaving;
        for (auto &j : admitted) {
            const bool resume = !j->acc.empty();
            int rc = CRK_OK;
            if (sv->prm.snapshot_every > 0) rc = j->snap_dev.ensure((size_t)j->n * 11 * sizeof(double));
            if (rc == CRK_OK)
                rc = pool_add(ln->sim, j->slot, j->phys, j->n, j->pos.data(), j->vel.data(), j->mass.data(),
                              j->u.data(), j->h.data(), j->sp.data(), resume ? j->acc.data() : nullptr,
                              resume ? j->du.data() : nullptr);
            std::lock_guard<std::mutex> lk(sv->mu);
            j->t_admit = clk::now();
            // a resumed job has the forces of its snapshot: no initial evaluation
            j->init_done = resume;
            if (rc != CRK_OK) {
                finish_locked(j, rc, crk_last_error());
                ln->slots[j->slot] = nullptr;
                sv->resident_bytes -= j->bytes;
            }
        }
        bool notify = false;
        // Cancelled jobs leave at this step boundary.
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            for (auto &j : ln->slots)
                if (j && !j->done && j->cancel) {
                    finish_locked(j, CRK_ECANCELED, "cancelled");
                    leaving.push_back(j);
                }
        }
        // A resumed job that already ran all its steps only publishes its state.
        for (auto &j : ln->slots) {
            if (!j) continue;
            bool ready;
            {
                std::lock_guard<std::mutex> lk(sv->mu);
                ready = !j->done && j->init_done && j->steps_done >= j->nsteps;
            }
            if (!ready) continue;
            Extracted e = extract(*ln, *j);
            std::lock_guard<std::mutex> lk(sv->mu);
            publish_locked(j, e);
            leaving.push_back(j);
        }
        // One batched step for every live resident job of the lane.
        bool any_live = false;
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            for (int s = 0; s < sv->prm.max_slots; ++s) {
                auto &j = ln->slots[s];
                const bool live = j && !j->done;
                dts[(size_t)s] = (live && j->init_done) ? j->dt : 0.0;
                any_live = any_live || live;
            }
        }
        int rc = any_live ? pool_step(ln->sim, dts.data()) : CRK_OK;
        if (rc != CRK_OK) {
            std::string msg = crk_last_error();
            std::lock_guard<std::mutex> lk(sv->mu);
            for (auto &j : ln->slots)
                if (j && !j->done) {
                    finish_locked(j, rc, msg.c_str());
                    leaving.push_back(j);
                }
        } else if (any_live) {
            for (auto &j : ln->slots) {
                bool finished;
                {
                    std::lock_guard<std::mutex> lk(sv->mu);
                    if (!j || j->done) continue;
                    if (!j->init_done) j->init_done = true;
                    else j->steps_done++;
                    const int every = sv->prm.snapshot_every;
                    if (every > 0 && j->steps_done > 0 && j->steps_done % every == 0) {
                        int r3 = start_snapshot(*ln, *j);
                        if (r3 != CRK_OK) {
                            finish_locked(j, r3, crk_last_error());
                            leaving.push_back(j);
                            continue;
                        }
                    }
                    finished = j->steps_done >= j->nsteps;
                }
                if (finished) {
                    Extracted e = extract(*ln, *j);
                    std::lock_guard<std::mutex> lk(sv->mu);
                    publish_locked(j, e);
                    leaving.push_back(j);
                }
            }
        }
        // a failed retirement launch leaves a CUDA error that the next step reports
        for (auto &j : leaving) (void)pool_remove(ln->sim, j->slot, j->n);
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            for (auto &j : leaving) {
                ln->slots[j->slot] = nullptr;
                sv->resident_bytes -= j->bytes;
                j->mass.clear();
                j->h.clear();
                j->sp.clear();
            }
            notify = !leaving.empty() || !admitted.empty();
        }
        if (notify) {
            sv->cv_done.notify_all();
            // freed budget may let another lane admit its queue head
            for (auto &other : sv->lanes)
                if (other.get() != ln) other->cv_work.notify_one();
        }
    }
}

void destroy_lane(Lane &ln)
{
    if (ln.side) cudaStreamSynchronize(ln.side);
    if (ln.sim) crk_destroy(ln.sim);
    if (ln.st) cudaStreamDestroy(ln.st);
    if (ln.side) cudaStreamDestroy(ln.side);
    if (ln.stepped) cudaEventDestroy(ln.stepped);
    ln.sim = nullptr;
    ln.st = ln.side = nullptr;
    ln.stepped = nullptr;
}

}  // namespace

extern "C" int crk_service_create(const crk_service_params *params, crk_service **out)
{
    if (!params || !out) return fail(CRK_EINVAL, "null argument");
    if (params->max_slots < 1 || params->max_slots > 65535)
        return fail(CRK_EINVAL, "max_slots must be in [1, 65535]");
    if (params->hbm_budget_bytes == 0) return fail(CRK_EINVAL, "hbm_budget_bytes must be > 0");
    if (params->snapshot_every < 0) return fail(CRK_EINVAL, "snapshot_every must be >= 0");
    if (params->size_classes < 0 || params->size_classes > kMaxClasses)
        return fail(CRK_EINVAL, "size_classes must be in [0, %d]", kMaxClasses);
    if (params->lane_priority < -1 || params->lane_priority > 1)
        return fail(CRK_EINVAL, "lane_priority must be -1, 0 or 1");
    CK(cudaSetDevice(params->device));
    auto *sv = new crk_service();
    sv->prm = *params;
    if (sv->prm.size_classes == 0) sv->prm.size_classes = kDefaultClasses;
    crk_params p{};
    p.kernel = CRK_WENDLAND_C4;
    p.leaf_cap = params->leaf_cap ? params->leaf_cap : 64;
    p.precision = params->precision;
    int rc = CRK_OK;
    // stream priorities: lower numbers run first; greatest <= least
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
        cudaGetLastError();
        least = greatest = 0;
    }
    const int K = sv->prm.size_classes;
    for (int k = 0; k < K && rc == CRK_OK; ++k) {
        auto ln = std::make_unique<Lane>();
        ln->index = k;
        int prio = least;
        if (sv->prm.lane_priority != 0 && K > 1) {
            const int rank = sv->prm.lane_priority > 0 ? k : K - 1 - k;   // 0 = lowest priority
            prio = least - (int)((long)(least - greatest) * rank / (K - 1));
        }
        cudaError_t e = cudaStreamCreateWithPriority(&ln->st, cudaStreamNonBlocking, prio);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ln->side, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ln->stepped, cudaEventDisableTiming);
        if (e != cudaSuccess) rc = fail(CRK_ECUDA, "stream creation failed: %s", cudaGetErrorString(e));
        if (rc == CRK_OK) rc = crk_create(&p, ln->st, &ln->sim);
        if (rc == CRK_OK) rc = pool_init(ln->sim, params->max_slots);
        ln->slots.assign((size_t)params->max_slots, nullptr);
        sv->lanes.push_back(std::move(ln));
    }
    if (rc != CRK_OK) {
        for (auto &ln : sv->lanes) destroy_lane(*ln);
        delete sv;
        return rc;
    }
    sv->bpp = pool_bytes_per_particle(sv->lanes[0]->sim);
    for (auto &ln : sv->lanes) ln->th = std::thread(worker, sv, ln.get());
    *out = sv;
    return CRK_OK;
}

extern "C" int crk_submit(crk_service *sv, const crk_job *job, uint64_t *ticket)
{
    if (!sv || !job || !ticket) return fail(CRK_EINVAL, "null argument");
    if (job->n <= 0 || !job->pos || !job->vel || !job->mass || !job->u || !job->h || !job->species)
        return fail(CRK_EINVAL, "a job needs n > 0 and every particle array");
    if (job->nsteps < 0 || !(job->dt >= 0.0)) return fail(CRK_EINVAL, "nsteps >= 0 and dt >= 0 required");
    const bool resume = job->acc != nullptr || job->dudt != nullptr || job->steps_done != 0;
    if (resume && (!job->acc || !job->dudt || job->steps_done < 0 || job->steps_done > job->nsteps))
        return fail(CRK_EINVAL, "a resumed job needs acc, dudt and 0 <= steps_done <= nsteps");
    auto j = std::make_shared<Job>();
    j->phys = job->phys;
    j->n = job->n;
    const size_t n = (size_t)job->n;
    j->bytes = n * (sv->bpp + (sv->prm.snapshot_every > 0 ? 11 * sizeof(double) : 0)) + (64u << 10);
    if (j->bytes > sv->prm.hbm_budget_bytes)
        return fail(CRK_EINVAL, "job of %lld particles needs %zu bytes, above the budget of %zu",
                    (long long)job->n, j->bytes, sv->prm.hbm_budget_bytes);
    int lane = 0;
    while (lane + 1 < sv->prm.size_classes && job->n >= class_bound(lane)) ++lane;
    j->lane = lane;
    j->pos.assign(job->pos, job->pos + 3 * n);
    j->vel.assign(job->vel, job->vel + 3 * n);
    j->mass.assign(job->mass, job->mass + n);
    j->u.assign(job->u, job->u + n);
    j->h.assign(job->h, job->h + n);
    j->sp.assign(job->species, job->species + n);
    if (resume) {
        j->acc.assign(job->acc, job->acc + 3 * n);
        j->du.assign(job->dudt, job->dudt + n);
        j->steps_done = job->steps_done;
    }
    j->dt = job->dt;
    j->nsteps = job->nsteps;
    if (sv->prm.snapshot_every > 0) {
        // the pinned host copy of the job's snapshots, on the service's device
        // (the caller's current device is restored)
        int prev = 0;
        cudaGetDevice(&prev);
        cudaSetDevice(sv->prm.device);
        cudaError_t e = cudaMallocHost(&j->snap_host, n * 11 * sizeof(double));
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j->snap_ev, cudaEventDisableTiming);
        cudaSetDevice(prev);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(CRK_ENOMEM, "no pinned memory or event for the snapshots of %lld particles",
                        (long long)job->n);
        }
    }
    j->t_submit = clk::now();
    Lane *ln = sv->lanes[(size_t)lane].get();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        j->ticket = sv->next_ticket++;
        sv->jobs[j->ticket] = j;
        ln->pending.push_back(j);
    }
    ln->cv_work.notify_one();
    *ticket = j->ticket;
    return CRK_OK;
}

extern "C" int crk_poll(crk_service *sv, uint64_t ticket, crk_job_result *res, int64_t timeout_us)
{
    if (!sv || !res) return fail(CRK_EINVAL, "null argument");
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->jobs.find(ticket);
    if (it == sv->jobs.end()) return fail(CRK_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    std::shared_ptr<Job> j = it->second;
    auto ready = [&] { return j->done; };
    if (timeout_us < 0) sv->cv_done.wait(lk, ready);
    else if (timeout_us > 0) sv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready);
    if (!j->done) return fail(CRK_EPENDING, "job %llu has not finished", (unsigned long long)ticket);
    sv->jobs.erase(it);
    // everything below was written under the mutex before done was set, and
    // the worker no longer touches a finished job's result
    lk.unlock();
    res->n = j->n;
    res->status = j->status;
    res->latency_ns = std::chrono::duration_cast<std::chrono::nanoseconds>(j->t_done - j->t_submit).count();
    res->queue_ns = std::chrono::duration_cast<std::chrono::nanoseconds>(j->t_admit - j->t_submit).count();
    if (j->status != CRK_OK) return fail(j->status, "job %llu failed: %s", (unsigned long long)ticket, j->msg.c_str());
    const size_t n = (size_t)j->n;
    if (res->pos) std::memcpy(res->pos, j->pos.data(), 3 * n * sizeof(double));
    if (res->vel) std::memcpy(res->vel, j->vel.data(), 3 * n * sizeof(double));
    if (res->u) std::memcpy(res->u, j->u.data(), n * sizeof(double));
    return CRK_OK;
}

extern "C" int crk_service_destroy(crk_service *sv)
{
    if (!sv) return CRK_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        // queued jobs that never started are cancelled
        for (auto &ln : sv->lanes) {
            for (auto &j : ln->pending) {
                j->t_admit = clk::now();
                finish_locked(j, CRK_EINVAL, "service destroyed before the job was admitted");
            }
            ln->pending.clear();
        }
    }
    for (auto &ln : sv->lanes) ln->cv_work.notify_all();
    for (auto &ln : sv->lanes)
        if (ln->th.joinable()) ln->th.join();
    sv->cv_done.notify_all();
    for (auto &ln : sv->lanes) destroy_lane(*ln);
    delete sv;
    return CRK_OK;
}

extern "C" int crk_service_snapshot(crk_service *sv, uint64_t ticket, crk_job_snapshot *out)
{
    if (!sv || !out) return fail(CRK_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->jobs.find(ticket);
    if (it == sv->jobs.end()) return fail(CRK_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    Job &j = *it->second;
    if (j.snap_inflight) {
        CK(cudaEventSynchronize(j.snap_ev));
        j.snap_valid = j.snap_steps;
        j.snap_inflight = false;
    }
    if (j.snap_valid < 0) return fail(CRK_EPENDING, "no snapshot of job %llu yet", (unsigned long long)ticket);
    const size_t n = (size_t)j.n;
    const double *b = j.snap_host;
    if (out->pos) std::memcpy(out->pos, b, 3 * n * sizeof(double));
    if (out->vel) std::memcpy(out->vel, b + 3 * n, 3 * n * sizeof(double));
    if (out->u) std::memcpy(out->u, b + 6 * n, n * sizeof(double));
    if (out->acc) std::memcpy(out->acc, b + 7 * n, 3 * n * sizeof(double));
    if (out->dudt) std::memcpy(out->dudt, b + 10 * n, n * sizeof(double));
    out->n = j.n;
    out->steps_done = j.snap_valid;
    return CRK_OK;
}

extern "C" int crk_service_cancel(crk_service *sv)
{
    if (!sv) return fail(CRK_EINVAL, "null argument");
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        for (auto &ln : sv->lanes) {
            for (auto &j : ln->pending) {
                j->t_admit = clk::now();
                finish_locked(j, CRK_ECANCELED, "cancelled before admission");
            }
            ln->pending.clear();
            for (auto &j : ln->slots)
                if (j) j->cancel = true;
        }
    }
    for (auto &ln : sv->lanes) ln->cv_work.notify_all();
    sv->cv_done.notify_all();
    return CRK_OK;
}
