// Batching and serving runtime of the sulfmg library.
//
// Batch: many independent domains (uneven sizes) advanced together.  Each of
// nstreams host workers owns a CUDA stream and takes the next instance (largest
// work first); an instance's multigrid cycles are its own captured CUDA graphs,
// so the GPU runs the kernels of several instances at once while each worker
// waits on its instance's convergence tests.  In lock-step mode the instances
// of one size class (same dimension, grid, levels, model-independent solver
// controls, dt and step count) form one work item: each phase of their cycles
// is one launch over all of them (solver.cu, lockstep.cu).
//
// Server: jobs (a level set, a model, a number of CN steps) are submitted at any
// time and admitted first-come-first-served among those whose device-memory
// estimate fits in what the budget has left; admitted jobs run on the worker
// streams as soon as a worker and memory are free (continuous batching), and
// their memory returns to the budget when they finish.  Latency is measured
// from submission to the moment the result is ready.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/sulfmg.h"
#include "sulf_internal.cuh"

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

// ---------------------------------------------------------------------------
// device-memory estimate of a domain (admission control)

extern "C" unsigned long long sulf_estimate_device_bytes(int dim, int N, int coarsest_N, int precision) {
    if ((dim != 2 && dim != 3) || N < 2 || coarsest_N < 2) return 0;
    double nn0 = 1;
    for (int a = 0; a < dim; a++) nn0 *= (double)(N + 1);
    // bytes per box node: FP64 level vectors (Wc, rhs, x, res 64; edges 16 dim;
    // 2x2 blocks and inverses 64, and their copies and rhs's in list order, at
    // most 80), geometry (phi, type, maps, lists, marks ~30), the finest
    // level's W^n, old-time part and staging (49); FP32 vectors (32 + 8 dim +
    // 32 + 32) when mixed; coarser levels add 1/(2^dim - 1)
    double per_level = 208.0 + 16.0 * dim + 30.0;
    if (precision == 1) per_level += 96.0 + 8.0 * dim;
    double geo = 1.0 / (1.0 - 1.0 / (double)(1 << dim));
    // ghost-row member tables: 3^dim members x (weight 8 + 4, node 4, ghost
    // index 4) per ghost, ghosts bounded by 8 % (2-D) / 15 % (3-D) of the box
    // nodes on every level (the coarse levels of thin 3-D shapes approach it)
    const double members = dim == 2 ? 9.0 : 27.0;
    per_level += (dim == 2 ? 0.08 : 0.15) * (members * 20.0 + 17.0 * dim);  // + orders, theta, normal
    // composed ghost relaxation: at most 24 (2-D) / 27 (3-D) entries per ghost
    // of 16 B (code 4, FP64 and FP32 weight) and the row pointer
    per_level += (dim == 2 ? 0.08 * (24.0 * 16.0 + 4.0) : 0.15 * (27.0 * 16.0 + 4.0));
    // band extension operator: 16 B per entry, at most 1.5 (2-D) / 3.2 (3-D)
    // entries per box node on any level
    per_level += (dim == 2 ? 1.5 : 3.2) * 16.0;
    double bytes = nn0 * (per_level * geo + 49.0);
    // ghost and band arrays, allocation granularity, coarsest dense matrices
    double nc = 1;
    for (int a = 0; a < dim; a++) nc *= (double)(coarsest_N + 1);
    double m = 2.0 * nc;
    bytes += 2.0 * m * m * 8.0 * (precision == 1 ? 1.5 : 1.0);
    bytes = bytes * 1.15 + 8.0 * 1024 * 1024;
    return (unsigned long long)bytes;
}

// ---------------------------------------------------------------------------
// batch

constexpr int kLockChunk = 32;  // instances per lock-step chunk (mode 1)

struct sulf_batch_s {
    std::vector<sulf_handle> h;
    std::vector<cudaStream_t> streams;
    std::vector<int> status;
    std::vector<std::string> errors;
    int device = 0;
    int lockstep = 0;
};

extern "C" int sulf_batch_create(const sulf_handle* handles, int n, int nstreams, sulf_batch* out) {
    if (!out) return sulf_fail(SULF_EINVAL, "out is NULL");
    *out = nullptr;
    if (!handles || n < 1 || nstreams < 1) return sulf_fail(SULF_EINVAL, "invalid arguments");
    for (int i = 0; i < n; i++)
        if (!handles[i]) return sulf_fail(SULF_EINVAL, "NULL handle in batch");
    sulf_batch b = new sulf_batch_s();
    b->h.assign(handles, handles + n);
    b->status.assign(n, SULF_OK);
    b->errors.assign(n, std::string());
    cudaGetDevice(&b->device);
    int ns = std::min(nstreams, n);
    for (int k = 0; k < ns; k++) {
        cudaStream_t s;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            sulf_batch_destroy(b);
            return sulf_fail(SULF_EDEVICE, "cannot create a CUDA stream");
        }
        b->streams.push_back(s);
    }
    *out = b;
    return SULF_OK;
}

extern "C" int sulf_batch_set_lockstep(sulf_batch b, int mode) {
    if (!b || mode < 0) return sulf_fail(SULF_EINVAL, "invalid arguments");
    b->lockstep = mode;
    return SULF_OK;
}

extern "C" int sulf_batch_step(sulf_batch b, const double* dt, const int* nsteps) {
    if (!b || !dt || !nsteps) return sulf_fail(SULF_EINVAL, "invalid arguments");
    const int n = (int)b->h.size();
    // work items: one instance, or (lock-step mode) a class of instances
    std::vector<std::vector<int>> items;
    if (b->lockstep) {
        std::vector<std::vector<double>> keys;
        for (int i = 0; i < n; i++) {
            std::vector<double> k;
            if (dt[i] > 0 && nsteps[i] > 0 && sulf::lockstep_key(b->h[i], k)) {
                k.push_back(dt[i]);
                k.push_back((double)nsteps[i]);
                size_t c = 0;
                while (c < keys.size() && keys[c] != k) c++;
                if (c == keys.size()) {
                    keys.push_back(k);
                    items.push_back({});
                }
                items[c].push_back(i);
            } else {
                items.push_back({i});
                keys.push_back({-1.0});  // matches no class key
            }
        }
    } else {
        for (int i = 0; i < n; i++) items.push_back({i});
    }
    std::vector<double> wi(n);
    for (int i = 0; i < n; i++) {
        sulf_stats st;
        sulf_get_stats(b->h[i], &st);
        wi[i] = (double)(st.n_inside + st.n_ghost) * nsteps[i];
    }
    if (b->lockstep) {
        // split the classes into chunks of at most `lockstep` instances
        // (mode 1: kLockChunk), dealt round-robin; the worker streams overlap
        // one chunk's host tests and per-instance set-up with the others'
        // cycles (on the 256-star batch, chunks of 32 ran 2-7 % faster than
        // of 8, of 64, or one chunk per stream)
        const int cap = b->lockstep >= 2 ? b->lockstep : kLockChunk;
        std::vector<std::vector<int>> split;
        for (auto& it : items) {
            const int k = (int)it.size();
            const int chunks = (k + cap - 1) / cap;
            for (int c = 0; c < chunks; c++) {
                split.push_back({});
                for (int q = c; q < k; q += chunks) split.back().push_back(it[q]);
            }
        }
        items.swap(split);
    }
    // largest work first: active nodes times steps
    std::vector<double> work(items.size(), 0.0);
    for (size_t j = 0; j < items.size(); j++)
        for (int i : items[j]) work[j] += wi[i];
    std::vector<size_t> order(items.size());
    for (size_t j = 0; j < order.size(); j++) order[j] = j;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t c) { return work[a] > work[c]; });
    std::atomic<int> next(0);
    auto worker = [&](int k) {
        cudaSetDevice(b->device);
        for (;;) {
            const int j = next.fetch_add(1);
            if (j >= (int)order.size()) break;
            const std::vector<int>& it = items[order[j]];
            if (it.size() == 1) {
                const int i = it[0];
                int rc = sulf_set_stream(b->h[i], b->streams[k]);
                if (rc == SULF_OK) rc = sulf_step(b->h[i], dt[i], nsteps[i]);
                b->status[i] = rc;
                b->errors[i] = rc ? sulf_last_error() : "";
                continue;
            }
            std::vector<sulf_handle> hs;
            for (int i : it) {
                sulf_set_stream(b->h[i], b->streams[k]);
                hs.push_back(b->h[i]);
            }
            std::vector<int> st(it.size(), SULF_OK);
            std::vector<std::string> err;
            int rc = sulf::lockstep_advance(hs.data(), (int)hs.size(), dt[it[0]], nsteps[it[0]], st.data(), err,
                                            b->streams[k]);
            const std::string cls = rc ? sulf_last_error() : "";
            for (size_t q = 0; q < it.size(); q++) {
                const int i = it[q];
                b->status[i] = rc ? rc : st[q];
                b->errors[i] = rc ? cls : err[q];
            }
        }
    };
    std::vector<std::thread> th;
    const int nw = std::min((int)b->streams.size(), (int)items.size());
    for (int k = 0; k < nw; k++) th.emplace_back(worker, k);
    for (auto& t : th) t.join();
    for (int i = 0; i < n; i++)
        if (b->status[i] != SULF_OK) return sulf_fail(b->status[i], "batch instance " + std::to_string(i) + ": " + b->errors[i]);
    return SULF_OK;
}

// tune each instance through the process cache: the first instance of a
// problem class is timed on the GPU alone (stream of worker 0), the others of
// the class take its result
extern "C" int sulf_batch_autotune(sulf_batch b, const double* dt, sulf_tune_result* out) {
    if (!b || !dt) return sulf_fail(SULF_EINVAL, "invalid arguments");
    for (size_t i = 0; i < b->h.size(); i++) {
        int rc = sulf_set_stream(b->h[i], b->streams[0]);
        sulf_tune_result r{};
        if (rc == SULF_OK) rc = sulf_autotune(b->h[i], dt[i], 1, &r);
        if (rc != SULF_OK) return rc;
        if (out) out[i] = r;
    }
    return SULF_OK;
}

extern "C" int sulf_batch_status(sulf_batch b, int* status) {
    if (!b || !status) return sulf_fail(SULF_EINVAL, "invalid arguments");
    for (size_t i = 0; i < b->status.size(); i++) status[i] = b->status[i];
    return SULF_OK;
}

extern "C" void sulf_batch_destroy(sulf_batch b) {
    if (!b) return;
    for (sulf_handle h : b->h) sulf_set_stream(h, nullptr);
    for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
    delete b;
}

// ---------------------------------------------------------------------------
// server

namespace {

struct Job {
    long long id = 0;
    sulf_job spec{};
    std::vector<double> phi;
    unsigned long long est = 0;
    double t_submit = 0, t_start = 0, t_done = 0;
    int status = SULF_OK;
    std::string err;
    std::vector<double> s, c;
    sulf_stats stats{};
    unsigned long long bytes = 0;
    bool done = false;
};

}  // namespace

struct sulf_server_s {
    unsigned long long budget = 0, reserved = 0, peak = 0;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Job*> queue;
    std::unordered_map<long long, Job*> jobs;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;
    bool stopping = false;
    long long next_id = 1, completed = 0, failed = 0, running = 0, max_running = 0;
    std::vector<double> latencies;
    double t_create = 0, t_last_done = 0;
};

namespace {

void run_job(Job* j, cudaStream_t stream) {
    const sulf_job& p = j->spec;
    double box[2] = {p.box_lo, p.box_hi};
    sulf_handle h = nullptr;
    int rc = sulf_create_domain(j->phi.data(), p.dim, box, p.N, p.coarsest_N, &h);
    if (rc == SULF_OK) rc = sulf_set_stream(h, stream);
    if (rc == SULF_OK) rc = sulf_set_model(h, &p.model);
    if (rc == SULF_OK) rc = sulf_set_solver(h, &p.solver);
    if (rc == SULF_OK) rc = sulf_step(h, p.dt, p.nsteps);
    if (rc == SULF_OK) {
        size_t nn = j->phi.size();
        j->s.resize(nn);
        j->c.resize(nn);
        rc = sulf_get_state(h, j->s.data(), j->c.data(), nullptr);
    }
    if (h) sulf_get_stats(h, &j->stats);
    j->status = rc;
    if (rc) j->err = sulf_last_error();
    if (h) {
        sulf_set_stream(h, nullptr);
        sulf_destroy(h);
    }
}

void server_worker(sulf_server s, int k) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        Job* pick = nullptr;
        for (auto it = s->queue.begin(); it != s->queue.end(); ++it)
            if (s->reserved + (*it)->est <= s->budget) {
                pick = *it;
                s->queue.erase(it);
                break;
            }
        if (!pick) {
            if (s->stopping && s->queue.empty()) return;
            s->cv_work.wait(lk);
            continue;
        }
        s->reserved += pick->est;
        s->peak = std::max(s->peak, s->reserved);
        s->running++;
        s->max_running = std::max(s->max_running, s->running);
        pick->t_start = now_ms();
        lk.unlock();
        run_job(pick, s->streams[k]);
        lk.lock();
        s->reserved -= pick->est;
        s->running--;
        pick->t_done = now_ms();
        s->t_last_done = pick->t_done;
        pick->done = true;
        if (pick->status == SULF_OK) {
            s->completed++;
            s->latencies.push_back(pick->t_done - pick->t_submit);
        } else {
            s->failed++;
        }
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
}

double percentile(std::vector<double> v, double q) {
    if (v.empty()) return 0;
    std::sort(v.begin(), v.end());
    double pos = q * (v.size() - 1);
    size_t lo = (size_t)pos, hi = std::min(lo + 1, v.size() - 1);
    return v[lo] + (pos - lo) * (v[hi] - v[lo]);
}

}  // namespace

extern "C" int sulf_server_create(unsigned long long budget_bytes, int nworkers, sulf_server* out) {
    if (!out) return sulf_fail(SULF_EINVAL, "out is NULL");
    *out = nullptr;
    if (budget_bytes == 0 || nworkers < 1) return sulf_fail(SULF_EINVAL, "invalid arguments");
    sulf_server s = new sulf_server_s();
    s->budget = budget_bytes;
    cudaGetDevice(&s->device);
    for (int k = 0; k < nworkers; k++) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            for (cudaStream_t t : s->streams) cudaStreamDestroy(t);
            delete s;
            return sulf_fail(SULF_EDEVICE, "cannot create a CUDA stream");
        }
        s->streams.push_back(st);
    }
    s->t_create = now_ms();
    for (int k = 0; k < nworkers; k++) s->workers.emplace_back(server_worker, s, k);
    *out = s;
    return SULF_OK;
}

extern "C" int sulf_server_submit(sulf_server s, const sulf_job* job, long long* id) {
    if (!s || !job || !id || !job->levelset || (job->dim != 2 && job->dim != 3) || job->N < 2 || job->nsteps < 0 ||
        !(job->dt > 0))
        return sulf_fail(SULF_EINVAL, "invalid job");
    Job* j = new Job();
    j->spec = *job;
    size_t nn = 1;
    for (int a = 0; a < job->dim; a++) nn *= (size_t)(job->N + 1);
    j->phi.assign(job->levelset, job->levelset + nn);
    j->spec.levelset = nullptr;
    j->est = sulf_estimate_device_bytes(job->dim, job->N, job->coarsest_N, job->solver.precision);
    if (j->est > s->budget) {
        delete j;
        return sulf_fail(SULF_ENOMEM, "job needs more device memory than the whole budget");
    }
    std::lock_guard<std::mutex> lk(s->mu);
    j->id = s->next_id++;
    j->t_submit = now_ms();
    s->jobs[j->id] = j;
    s->queue.push_back(j);
    *id = j->id;
    s->cv_work.notify_one();
    return SULF_OK;
}

extern "C" int sulf_server_poll(sulf_server s, long long id, int* done) {
    if (!s || !done) return sulf_fail(SULF_EINVAL, "invalid arguments");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(id);
    if (it == s->jobs.end()) return sulf_fail(SULF_EINVAL, "unknown job id");
    *done = it->second->done ? 1 : 0;
    return SULF_OK;
}

extern "C" int sulf_server_wait(sulf_server s, long long id, double* s_out, double* c_out, sulf_job_result* res) {
    if (!s) return sulf_fail(SULF_EINVAL, "invalid arguments");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(id);
    if (it == s->jobs.end()) return sulf_fail(SULF_EINVAL, "unknown job id");
    Job* j = it->second;
    s->cv_done.wait(lk, [&] { return j->done; });
    s->jobs.erase(it);
    lk.unlock();
    if (res) {
        res->status = j->status;
        res->latency_ms = j->t_done - j->t_submit;
        res->queue_ms = j->t_start - j->t_submit;
        res->run_ms = j->t_done - j->t_start;
        res->estimate_bytes = j->est;
        res->device_bytes = j->stats.device_bytes;
        res->newton = j->stats.newton_total;
        res->cycles = j->stats.cycles_total;
    }
    int rc = j->status;
    if (rc == SULF_OK) {
        if (s_out) std::copy(j->s.begin(), j->s.end(), s_out);
        if (c_out) std::copy(j->c.begin(), j->c.end(), c_out);
    }
    std::string err = j->err;
    delete j;
    if (rc) return sulf_fail(rc, err);
    return SULF_OK;
}

extern "C" int sulf_server_get_stats(sulf_server s, sulf_server_stats* out) {
    if (!s || !out) return sulf_fail(SULF_EINVAL, "invalid arguments");
    std::lock_guard<std::mutex> lk(s->mu);
    out->completed = s->completed;
    out->failed = s->failed;
    out->queued = (long long)s->queue.size();
    out->running = s->running;
    out->max_running = s->max_running;
    out->p50_ms = percentile(s->latencies, 0.50);
    out->p99_ms = percentile(s->latencies, 0.99);
    out->budget_bytes = s->budget;
    out->peak_reserved_bytes = s->peak;
    double span = (s->t_last_done - s->t_create) / 1e3;
    out->jobs_per_s = span > 0 ? s->completed / span : 0;
    return SULF_OK;
}

extern "C" void sulf_server_destroy(sulf_server s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
    }
    s->cv_work.notify_all();
    for (auto& t : s->workers) t.join();
    for (auto& kv : s->jobs) delete kv.second;
    for (cudaStream_t t : s->streams) cudaStreamDestroy(t);
    delete s;
}
