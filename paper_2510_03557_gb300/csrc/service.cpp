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
    std::vector<uint8_t> sp;
    double dt = 0.0;
    int nsteps = 0;
    int steps_done = 0;
    bool init_done = false;
    int slot = -1;
    size_t bytes = 0;
    int status = CRK_OK;
    std::string msg;
    bool done = false;
    clk::time_point t_submit, t_admit, t_done;
};

}  // namespace

struct crk_service {
    crk_service_params prm{};
    crk_sim *sim = nullptr;
    cudaStream_t st = nullptr;
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
            int rc = pool_add(sv->sim, j->slot, j->phys, j->n, j->pos.data(), j->vel.data(),
                              j->mass.data(), j->u.data(), j->h.data(), j->sp.data());
            j->t_admit = clk::now();
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
        // One batched step for every resident job.
        for (int s = 0; s < sv->prm.max_slots; ++s) {
            auto &j = sv->slots[s];
            dts[(size_t)s] = (j && j->init_done) ? j->dt : 0.0;
        }
        int rc = pool_step(sv->sim, dts.data());
        std::vector<std::shared_ptr<Job>> leaving;
        if (rc != CRK_OK) {
            std::string msg = crk_last_error();
            for (auto &j : sv->slots)
                if (j && !j->done) {
                    finish(sv, j, rc, msg.c_str());
                    leaving.push_back(j);
                }
        } else {
            for (auto &j : sv->slots) {
                if (!j || j->done) continue;
                if (!j->init_done) j->init_done = true;
                else j->steps_done++;
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
    CK(cudaSetDevice(params->device));
    auto *sv = new crk_service();
    sv->prm = *params;
    crk_params p{};
    p.kernel = CRK_WENDLAND_C4;
    p.leaf_cap = params->leaf_cap ? params->leaf_cap : 64;
    p.precision = params->precision;
    cudaError_t e = cudaStreamCreateWithFlags(&sv->st, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete sv;
        return fail(CRK_ECUDA, "stream creation failed: %s", cudaGetErrorString(e));
    }
    int rc = crk_create(&p, sv->st, &sv->sim);
    if (rc == CRK_OK) rc = pool_init(sv->sim, params->max_slots);
    if (rc != CRK_OK) {
        if (sv->sim) crk_destroy(sv->sim);
        cudaStreamDestroy(sv->st);
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
    j->dt = job->dt;
    j->nsteps = job->nsteps;
    j->bytes = n * sv->bpp + (64u << 10);
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
    crk_destroy(sv->sim);
    cudaStreamDestroy(sv->st);
    delete sv;
    return CRK_OK;
}
