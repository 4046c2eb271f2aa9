// Continuous-batching service for many small-box force-and-KDK jobs (the
// shape of an emulator campaign).  One host thread owns a pool handle whose
// box slots hold the resident jobs' particles and trees on the device; each
// iteration it admits queued jobs into free slots while the HBM budget
// allows, advances every resident job by one KDK step in the same batched
// launches (a newly admitted job's first step is its initial force
// evaluation, dt = 0), and publishes jobs whose steps are done.  The
// paper's GPU-resident design (Sec. IV-A: data stays on the device for the
// whole PM step) applied across jobs instead of across substeps.
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

struct Job {
    uint64_t ticket = 0;
    crk_physics phys{};
    int64_t n = 0;
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
    // snapshot: device staging (11 n doubles), pinned host copy, completion event
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

}  // namespace

struct crk_service {
    crk_service_params prm{};
    crk_sim *sim = nullptr;
    cudaStream_t st = nullptr;
    cudaStream_t side = nullptr;  // snapshot copies
    cudaEvent_t stepped = nullptr;
    size_t bpp = 0;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Job>> pending;
    std::vector<std::shared_ptr<Job>> slots;
    std::unordered_map<uint64_t, std::shared_ptr<Job>> jobs;
    uint64_t next_ticket = 1;
    size_t resident_bytes = 0;
    bool stop = false;
};

namespace {

// Starts a snapshot of a resident job: extraction on the compute stream,
// device-to-host copy on the side stream (overlapping the next step).  The
// previous copy of the job is completed first (its staging is reused).
// Caller holds sv->mu.
int start_snapshot(crk_service *sv, Job &j)
{
    const size_t words = (size_t)j.n * 11;
    if (!j.snap_host) {
        if (cudaMallocHost(&j.snap_host, words * sizeof(double)) != cudaSuccess) {
            j.snap_host = nullptr;
            return fail(CRK_ENOMEM, "no pinned memory for a snapshot of %lld particles", (long long)j.n);
        }
        CK(cudaEventCreateWithFlags(&j.snap_ev, cudaEventDisableTiming));
    }
    if (j.snap_inflight) {
        CK(cudaEventSynchronize(j.snap_ev));
        j.snap_valid = j.snap_steps;
        j.snap_inflight = false;
    }
    RET(j.snap_dev.ensure(words * sizeof(double)));
    RET(pool_snapshot(sv->sim, j.slot, j.n, j.snap_dev.as<double>()));
    CK(cudaEventRecord(sv->stepped, sv->st));
    CK(cudaStreamWaitEvent(sv->side, sv->stepped, 0));
    CK(cudaMemcpyAsync(j.snap_host, j.snap_dev.p, words * sizeof(double), cudaMemcpyDeviceToHost, sv->side));
    CK(cudaEventRecord(j.snap_ev, sv->side));
    j.snap_steps = j.steps_done;
    j.snap_inflight = true;
    return CRK_OK;
}

void finish(crk_service *sv, const std::shared_ptr<Job> &j, int status, const char *msg)
{
    j->status = status;
    if (msg) j->msg = msg;
    j->t_done = clk::now();
    j->done = true;
}

void worker(crk_service *sv)
{
    cudaSetDevice(sv->prm.device);
    std::vector<double> dts((size_t)sv->prm.max_slots, 0.0);
    while (true) {
        std::vector<std::shared_ptr<Job>> admitted;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            // FIFO admission while a slot and the budget allow.
            while (!sv->pending.empty()) {
                auto &j = sv->pending.front();
                int free_slot = -1;
                for (int s = 0; s < sv->prm.max_slots; ++s)
                    if (!sv->slots[s]) {
                        free_slot = s;
                        break;
                    }
                if (free_slot < 0 || sv->resident_bytes + j->bytes > sv->prm.hbm_budget_bytes) break;
                j->slot = free_slot;
                sv->slots[free_slot] = j;
                sv->resident_bytes += j->bytes;
                admitted.push_back(j);
                sv->pending.pop_front();
            }
            bool any = false;
            for (auto &p : sv->slots) any = any || (p != nullptr);
            if (!any) {
                if (sv->stop) break;
                sv->cv_work.wait(lk);
                continue;
            }
        }
        std::vector<std::shared_ptr<Job>> published;
        for (auto &j : admitted) {
            const bool resume = !j->acc.empty();
            int rc = pool_add(sv->sim, j->slot, j->phys, j->n, j->pos.data(), j->vel.data(),
                              j->mass.data(), j->u.data(), j->h.data(), j->sp.data(),
                              resume ? j->acc.data() : nullptr, resume ? j->du.data() : nullptr);
            j->t_admit = clk::now();
            // a resumed job has the forces of its snapshot: no initial evaluation
            j->init_done = resume;
            if (rc != CRK_OK) {
                finish(sv, j, rc, crk_last_error());
                published.push_back(j);
            }
        }
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            for (auto &j : published) {
                sv->slots[j->slot] = nullptr;
                sv->resident_bytes -= j->bytes;
            }
        }
        std::vector<std::shared_ptr<Job>> leaving;
        // Cancelled jobs leave at this step boundary.
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            for (auto &j : sv->slots)
                if (j && !j->done && j->cancel) {
                    finish(sv, j, CRK_ECANCELED, "cancelled");
                    leaving.push_back(j);
                }
        }
        // A resumed job that already ran all its steps only publishes its state.
        for (auto &j : sv->slots)
            if (j && !j->done && j->init_done && j->steps_done >= j->nsteps) {
                std::vector<double> pos((size_t)j->n * 3), vel((size_t)j->n * 3), u((size_t)j->n);
                int r2 = pool_extract(sv->sim, j->slot, j->n, pos.data(), vel.data(), u.data());
                j->pos.swap(pos);
                j->vel.swap(vel);
                j->u.swap(u);
                finish(sv, j, r2, r2 == CRK_OK ? nullptr : crk_last_error());
                leaving.push_back(j);
            }
        // One batched step for every resident job.
        for (int s = 0; s < sv->prm.max_slots; ++s) {
            auto &j = sv->slots[s];
            dts[(size_t)s] = (j && !j->done && j->init_done) ? j->dt : 0.0;
        }
        bool any_live = false;
        for (auto &j : sv->slots) any_live = any_live || (j && !j->done);
        int rc = any_live ? pool_step(sv->sim, dts.data()) : CRK_OK;
        if (rc != CRK_OK) {
            std::string msg = crk_last_error();
            for (auto &j : sv->slots)
                if (j && !j->done) {
                    finish(sv, j, rc, msg.c_str());
                    leaving.push_back(j);
                }
        } else if (any_live) {
            for (auto &j : sv->slots) {
                if (!j || j->done) continue;
                if (!j->init_done) j->init_done = true;
                else j->steps_done++;
                const int every = sv->prm.snapshot_every;
                if (every > 0 && j->steps_done > 0 && j->steps_done % every == 0) {
                    std::lock_guard<std::mutex> lk(sv->mu);
                    int r3 = start_snapshot(sv, *j);
                    if (r3 != CRK_OK) {
                        finish(sv, j, r3, crk_last_error());
                        leaving.push_back(j);
                        continue;
                    }
                }
                if (j->steps_done >= j->nsteps) {
                    std::vector<double> pos((size_t)j->n * 3), vel((size_t)j->n * 3), u((size_t)j->n);
                    int r2 = pool_extract(sv->sim, j->slot, j->n, pos.data(), vel.data(), u.data());
                    j->pos.swap(pos);
                    j->vel.swap(vel);
                    j->u.swap(u);
                    finish(sv, j, r2, r2 == CRK_OK ? nullptr : crk_last_error());
                    leaving.push_back(j);
                }
            }
        }
        // a failed retirement launch leaves a CUDA error that the next step reports
        for (auto &j : leaving) (void)pool_remove(sv->sim, j->slot, j->n);
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            for (auto &j : leaving) {
                sv->slots[j->slot] = nullptr;
                sv->resident_bytes -= j->bytes;
                j->mass.clear();
                j->h.clear();
                j->sp.clear();
            }
        }
        if (!leaving.empty() || !published.empty()) sv->cv_done.notify_all();
    }
}

}  // namespace

extern "C" int crk_service_create(const crk_service_params *params, crk_service **out)
{
    if (!params || !out) return fail(CRK_EINVAL, "null argument");
    if (params->max_slots < 1 || params->max_slots > 65535)
        return fail(CRK_EINVAL, "max_slots must be in [1, 65535]");
    if (params->hbm_budget_bytes == 0) return fail(CRK_EINVAL, "hbm_budget_bytes must be > 0");
    if (params->snapshot_every < 0) return fail(CRK_EINVAL, "snapshot_every must be >= 0");
    CK(cudaSetDevice(params->device));
    auto *sv = new crk_service();
    sv->prm = *params;
    crk_params p{};
    p.kernel = CRK_WENDLAND_C4;
    p.leaf_cap = params->leaf_cap ? params->leaf_cap : 64;
    p.precision = params->precision;
    cudaError_t e = cudaStreamCreateWithFlags(&sv->st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sv->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sv->stepped, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        if (sv->st) cudaStreamDestroy(sv->st);
        if (sv->side) cudaStreamDestroy(sv->side);
        delete sv;
        return fail(CRK_ECUDA, "stream creation failed: %s", cudaGetErrorString(e));
    }
    int rc = crk_create(&p, sv->st, &sv->sim);
    if (rc == CRK_OK) rc = pool_init(sv->sim, params->max_slots);
    if (rc != CRK_OK) {
        if (sv->sim) crk_destroy(sv->sim);
        cudaStreamDestroy(sv->st);
        cudaStreamDestroy(sv->side);
        cudaEventDestroy(sv->stepped);
        delete sv;
        return rc;
    }
    sv->bpp = pool_bytes_per_particle(sv->sim);
    sv->slots.assign((size_t)params->max_slots, nullptr);
    sv->th = std::thread(worker, sv);
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
    j->bytes = n * (sv->bpp + (sv->prm.snapshot_every > 0 ? 11 * sizeof(double) : 0)) + (64u << 10);
    if (j->bytes > sv->prm.hbm_budget_bytes)
        return fail(CRK_EINVAL, "job of %lld particles needs %zu bytes, above the budget of %zu",
                    (long long)job->n, j->bytes, sv->prm.hbm_budget_bytes);
    j->t_submit = clk::now();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        j->ticket = sv->next_ticket++;
        sv->jobs[j->ticket] = j;
        sv->pending.push_back(j);
    }
    sv->cv_work.notify_one();
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
        for (auto &j : sv->pending) {
            j->status = CRK_EINVAL;
            j->msg = "service destroyed before the job was admitted";
            j->done = true;
        }
        sv->pending.clear();
    }
    sv->cv_work.notify_all();
    if (sv->th.joinable()) sv->th.join();
    sv->cv_done.notify_all();
    cudaStreamSynchronize(sv->side);
    crk_destroy(sv->sim);
    cudaStreamDestroy(sv->st);
    cudaStreamDestroy(sv->side);
    cudaEventDestroy(sv->stepped);
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
        for (auto &j : sv->pending) {
            j->status = CRK_ECANCELED;
            j->msg = "cancelled before admission";
            j->t_admit = j->t_done = clk::now();
            j->done = true;
        }
        sv->pending.clear();
        for (auto &j : sv->slots)
            if (j) j->cancel = true;
    }
    sv->cv_work.notify_all();
    sv->cv_done.notify_all();
    return CRK_OK;
}
