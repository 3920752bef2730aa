// Lattice server: jobs (one lattice each: parameters, initial fields, step count) are submitted
// from any host thread and run by one worker thread that keeps every admitted job in one
// many-lattice batch (continuous batching): each round advances all active jobs by one chunk of
// steps, finished jobs leave with their final fields copied out, and queued jobs join at the
// next round.  Job workspaces are carved from one caller-owned device arena.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "lbm_internal.h"
#include "serve_sched.h"

using namespace lbm_host;

namespace {

struct ServerJob {
    lbm_params prm;
    const double* in[5];
    double* out[5];
    int64_t steps, cells;
    size_t bytes;
    double t_submit, t_admit;
    lbm_handle* h;
};

}  // namespace

struct lbm_server {
    int device;
    cudaStream_t stream;
    char* job_arena;
    lbm_server_config cfg;
    lbm_serve::Scheduler* sched;
    lbm_batch* batch;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop;
    int fatal;               // sticky error of the worker (LBM_OK while healthy)
    std::string fatal_msg;
    std::unordered_map<int64_t, ServerJob> jobs;
    int64_t next_id;
    std::deque<lbm_job_result> results;
    std::chrono::steady_clock::time_point t0;
    lbm_server_stats st;
    int64_t other_launches;  // init and moments kernels of the jobs
};

namespace {

double now_s(const lbm_server* s) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

void post_result(lbm_server* s, const ServerJob& j, int64_t id, int status, const char* msg, double t_done) {
    lbm_job_result r;
    std::memset(&r, 0, sizeof(r));
    r.id = id;
    r.status = status;
    r.storage = j.prm.storage;
    r.nx = j.prm.nx;
    r.ny = j.prm.ny;
    r.steps = j.steps;
    r.t_submit = j.t_submit;
    r.t_admit = j.t_admit;
    r.t_done = t_done;
    if (msg) std::snprintf(r.message, sizeof(r.message), "%s", msg);
    s->results.push_back(r);
    s->st.completed++;
}

// Copy out and free a finished (or failed) job; called by the worker without the lock held.
void retire(lbm_server* s, int64_t id, ServerJob* j, int status_in) {
    int status = status_in;
    std::string msg = status ? g_err : std::string();
    if (j->h) {
        if (!status) {
            status = lbm_status(j->h);
            if (status) msg = g_err;
        }
        unsigned mask = 0;
        for (int k = 0; k < 5; ++k)
            if (j->out[k]) mask |= 1u << k;
        if (mask && status != LBM_ECUDA) {
            int rc = lbm_get_moments(j->h, mask, j->out, LBM_MEM_HOST);
            s->other_launches++;
            if (rc && !status) {
                status = rc;
                msg = g_err;
            }
        }
        lbm_destroy(j->h);
        j->h = nullptr;
    }
    const double t = now_s(s);
    std::lock_guard<std::mutex> lk(s->mu);
    post_result(s, *j, id, status, msg.c_str(), t);
    s->jobs.erase(id);
    s->cv_done.notify_all();
}

void worker_main(lbm_server* s) {
    cudaSetDevice(s->device);
    bool changed = false;
    for (;;) {
        std::vector<lbm_serve::Admit> adm;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stop || !s->sched->idle() || s->sched->queued() > 0; });
            if (s->stop) break;
            adm = s->sched->admit();
            const double t = now_s(s);
            for (const auto& a : adm) s->jobs[a.id].t_admit = t;
        }
        // create and initialise the admitted jobs
        for (const auto& a : adm) {
            ServerJob* j;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                j = &s->jobs[a.id];
            }
            int rc = lbm_create(&j->prm, s->job_arena + a.offset, j->bytes, s->stream, &j->h);
            if (!rc) {
                rc = lbm_init_fields(j->h, j->in[0], j->in[1], j->in[2], j->in[3], j->in[4], LBM_MEM_HOST);
                s->other_launches++;
            }
            if (rc) {
                {
                    std::lock_guard<std::mutex> lk(s->mu);
                    s->sched->cancel(a.id);
                }
                retire(s, a.id, j, rc);
                continue;
            }
            changed = true;
        }
        std::vector<int64_t> ids;
        int64_t n = 0;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            ids = s->sched->active_ids();
            n = s->sched->next_chunk(s->cfg.chunk_steps);
        }
        if (changed) {
            std::vector<lbm_handle*> members;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                for (int64_t id : ids) members.push_back(s->jobs[id].h);
            }
            int rc = lbm_batch_set_members(s->batch, members.data(), (int)members.size());
            if (rc) {
                std::lock_guard<std::mutex> lk(s->mu);
                s->fatal = rc;
                s->fatal_msg = g_err;
                break;
            }
            changed = false;
        }
        if (n <= 0) continue;
        const auto t_round = std::chrono::steady_clock::now();
        int rc = lbm_batch_step(s->batch, n);
        if (!rc && cudaStreamSynchronize(s->stream) != cudaSuccess)
            rc = fail(LBM_ECUDA, "worker stream: %s", cudaGetErrorString(cudaGetLastError()));
        if (rc) {
            std::lock_guard<std::mutex> lk(s->mu);
            s->fatal = rc;
            s->fatal_msg = g_err;
            break;
        }
        std::vector<int64_t> fin;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            int64_t cells = 0;
            for (int64_t id : ids) cells += s->jobs[id].cells;
            s->st.lattice_updates += cells * n;
            s->st.rounds++;
            s->st.busy_seconds += std::chrono::duration<double>(std::chrono::steady_clock::now() - t_round).count();
            fin = s->sched->advance(n);
        }
        for (int64_t id : fin) {
            ServerJob* j;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                j = &s->jobs[id];
            }
            retire(s, id, j, LBM_OK);
            changed = true;
        }
    }
    // stopping (or fatal): fail what is still active or queued
    std::vector<int64_t> left;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (auto& kv : s->jobs) left.push_back(kv.first);
    }
    if (s->batch) lbm_batch_set_members(s->batch, nullptr, 0);
    for (int64_t id : left) {
        ServerJob* j;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            j = &s->jobs[id];
            s->sched->cancel(id);
        }
        g_err = s->fatal ? s->fatal_msg : std::string("server stopped before the job finished");
        retire(s, id, j, s->fatal ? s->fatal : LBM_ESTATE);
    }
    std::lock_guard<std::mutex> lk(s->mu);
    s->cv_done.notify_all();
}

}  // namespace

extern "C" {

int lbm_server_workspace_bytes(const lbm_server_config* cfg, size_t job_arena_bytes, size_t* bytes) {
    g_err.clear();
    if (!cfg || !bytes) return fail(LBM_EINVAL, "NULL argument");
    size_t b = 0;
    int rc = lbm_batch_workspace_bytes(cfg->max_jobs, cfg->max_tiles, &b);
    if (rc) return rc;
    *bytes = align_up(b) + align_up(job_arena_bytes);
    return LBM_OK;
}

int lbm_server_create(const lbm_server_config* cfg, void* d_workspace, size_t bytes, void* cuda_stream,
                      lbm_server** out) {
    g_err.clear();
    if (!cfg || !out) return fail(LBM_EINVAL, "NULL argument");
    *out = nullptr;
    if (cfg->policy != LBM_SERVE_FCFS && cfg->policy != LBM_SERVE_SHORTEST_FIRST) return fail(LBM_EINVAL, "bad policy");
    if (cfg->max_jobs < 1 || cfg->max_cells < 1 || cfg->max_tiles < 1 || cfg->chunk_steps < 1)
        return fail(LBM_EINVAL, "max_jobs, max_cells, max_tiles and chunk_steps must be >= 1");
    if (!cuda_stream) return fail(LBM_EINVAL, "the server needs a created CUDA stream (not the legacy default stream)");
    size_t bb = 0;
    int rc = lbm_batch_workspace_bytes(cfg->max_jobs, cfg->max_tiles, &bb);
    if (rc) return rc;
    bb = align_up(bb);
    if (!d_workspace || reinterpret_cast<uintptr_t>(d_workspace) % kAlign)
        return fail(LBM_EINVAL, "workspace NULL or not 256-byte aligned");
    if (bytes <= bb) return fail(LBM_ENOMEM, "workspace of %zu bytes leaves no job arena", bytes);
    int device = 0;
    LBM_CUDA(cudaGetDevice(&device));
    lbm_server* s = new (std::nothrow) lbm_server;
    if (!s) return fail(LBM_ENOMEM, "host allocation failed");
    s->device = device;
    s->stream = static_cast<cudaStream_t>(cuda_stream);
    s->cfg = *cfg;
    s->job_arena = static_cast<char*>(d_workspace) + bb;
    s->sched = new lbm_serve::Scheduler(cfg->policy == LBM_SERVE_SHORTEST_FIRST ? lbm_serve::kShortestFirst
                                                                                 : lbm_serve::kFCFS,
                                        cfg->max_jobs, cfg->max_cells, cfg->max_tiles, bytes - bb);
    s->batch = nullptr;
    s->stop = false;
    s->fatal = LBM_OK;
    s->next_id = 1;
    s->t0 = std::chrono::steady_clock::now();
    std::memset(&s->st, 0, sizeof(s->st));
    s->other_launches = 0;
    rc = lbm_batch_create(cfg->max_jobs, cfg->max_tiles, d_workspace, bb, cuda_stream, &s->batch);
    if (!rc) rc = lbm_batch_set_schedule(s->batch, cfg->schedule, cfg->graph_steps);
    if (rc) {
        if (s->batch) lbm_batch_destroy(s->batch);
        delete s->sched;
        delete s;
        return rc;
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return LBM_OK;
}

int lbm_server_submit(lbm_server* s, const lbm_params* p, const double* phi, const double* psi, const double* ux,
                      const double* uy, const double* P, int64_t steps, double* const out[5], int64_t* id) {
    g_err.clear();
    if (!s || !p || !id) return fail(LBM_EINVAL, "NULL argument");
    if (!phi || !psi || !ux || !uy || !P) return fail(LBM_EINVAL, "all five fields are required");
    if (steps < 1) return fail(LBM_EINVAL, "steps must be >= 1");
    size_t bytes = 0;
    int rc = lbm_workspace_bytes(p, &bytes);
    if (rc) return rc;
    ServerJob j;
    std::memset(&j, 0, sizeof(j));
    j.prm = *p;
    j.in[0] = phi; j.in[1] = psi; j.in[2] = ux; j.in[3] = uy; j.in[4] = P;
    for (int k = 0; k < 5; ++k) j.out[k] = out ? out[k] : nullptr;
    j.steps = steps;
    j.cells = (int64_t)p->nx * p->ny;
    j.bytes = bytes;
    const lbm::TileDims td = lbm::tile_dims(p->storage);
    const int64_t tiles = (int64_t)((p->nx + td.tx - 1) / td.tx) * ((p->ny + td.ty - 1) / td.ty);
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->fatal) return fail(s->fatal, "server failed: %s", s->fatal_msg.c_str());
    if (s->stop) return fail(LBM_ESTATE, "server is stopping");
    const int64_t jid = s->next_id;
    j.t_submit = now_s(s);
    if (!s->sched->submit(lbm_serve::JobSpec{jid, j.cells, tiles, steps, bytes}))
        return fail(LBM_EINVAL, "job of %zu bytes / %lld tiles can never fit the server (arena %zu bytes, max_tiles %lld)",
                    bytes, (long long)tiles, s->sched->arena().size(), (long long)s->cfg.max_tiles);
    s->next_id++;
    s->jobs[jid] = j;
    s->st.submitted++;
    *id = jid;
    s->cv_work.notify_one();
    return LBM_OK;
}

int lbm_server_poll(lbm_server* s, lbm_job_result* out, int max, double timeout_s, int* n) {
    g_err.clear();
    if (!s || !n || (max > 0 && !out)) return fail(LBM_EINVAL, "NULL argument");
    *n = 0;
    std::unique_lock<std::mutex> lk(s->mu);
    if (timeout_s > 0 && s->results.empty() && !s->fatal)
        s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return !s->results.empty() || s->fatal; });
    while (*n < max && !s->results.empty()) {
        out[(*n)++] = s->results.front();
        s->results.pop_front();
    }
    if (s->fatal && s->results.empty() && *n == 0) return fail(s->fatal, "server failed: %s", s->fatal_msg.c_str());
    return LBM_OK;
}

int lbm_server_get_stats(lbm_server* s, lbm_server_stats* out) {
    g_err.clear();
    if (!s || !out) return fail(LBM_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->st;
    out->queued = (int64_t)s->sched->queued();
    out->active = (int64_t)s->sched->active_count();
    out->now = now_s(s);
    int64_t bl = 0;
    lbm_batch_launches(s->batch, &bl);
    out->kernel_launches = bl + s->other_launches;
    return LBM_OK;
}

int lbm_server_destroy(lbm_server* s) {
    g_err.clear();
    if (!s) return LBM_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    int rc = lbm_batch_destroy(s->batch);
    delete s->sched;
    delete s;
    return rc;
}

}  // extern "C"
