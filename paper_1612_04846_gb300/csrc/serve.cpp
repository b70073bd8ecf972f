// Continuous-batching solve server over the plan API (declared in bura.h).
//
// Requests arrive from any thread and wait in one FIFO queue.  Worker threads, each with its own
// non-blocking CUDA stream, take them in arrival order.  Plans stay resident between requests in a
// pool keyed by class (grid, coefficient field, k): an idle plan of the request's class is reused,
// moved to the request's alpha by bura_retarget when it differs (a host Remez solve and small table
// copies; the hierarchy, tensor maps and captured PCG graph stay).  Without one, the worker sets up a
// new plan if the resident plans plus the new one's estimated size fit the memory budget, after
// evicting idle plans of other classes in least-recently-used order; otherwise it waits until a plan
// becomes idle.  Each plan serves one request at a time, so requests of one class run concurrently
// on separate plans.  The Remez solves of new alphas run on the worker threads, overlapping the
// solves of the other workers on the GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "bura.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct PlanClass {
    int dim, n0, n1, n2, coef_kind, k;
    unsigned long long field;
    bool operator==(const PlanClass& o) const {
        return dim == o.dim && n0 == o.n0 && n1 == o.n1 && n2 == o.n2 && coef_kind == o.coef_kind && k == o.k &&
               field == o.field;
    }
};

PlanClass class_of(const bura_request& r) {
    PlanClass c;
    c.dim = r.grid.dim;
    c.n0 = r.grid.n[0];
    c.n1 = r.grid.n[1];
    c.n2 = r.grid.dim == 3 ? r.grid.n[2] : 1;
    c.coef_kind = r.grid.coef_kind;
    c.k = r.k;
    c.field = r.grid.coef_kind == BURA_COEF_FACES ? r.field : 0ull;
    return c;
}

long long points_of(const bura_grid& g) {
    long long n = 1;
    for (int a = 0; a < g.dim; ++a) n *= g.n[a];
    return n;
}

// Device bytes of a plan before it exists, from its buffers: the finest level holds 9 multi-shift vectors
// of the inner precision (x, r, two directions, q, and b, two iterates, a Chebyshev direction) and
// every coarser level 4, so 9 + 4/3 (2-D) or 9 + 4/7 (3-D) finest-level vectors in all, plus the two
// FP64 refinement vectors of the mixed path.  Replaced by the measured size of the first plan of the
// class.
size_t estimate_bytes(const bura_request& r, const bura_options& o) {
    const double N = (double)points_of(r.grid);
    const double K = r.k + 1;
    const double kp32 = 4.0 * std::ceil(K / 4.0), kp64 = 2.0 * std::ceil(K / 2.0);
    const double vecs = 9.0 + (r.grid.dim == 3 ? 4.0 / 7.0 : 4.0 / 3.0);
    double b = o.precision == BURA_PREC_MIXED ? N * (vecs * kp32 * 4.0 + 2.0 * kp64 * 8.0) : N * (vecs + 2.0) * kp64 * 8.0;
    if (r.grid.coef_kind == BURA_COEF_FACES) b += N * r.grid.dim * 8.0 * 3.0;
    return (size_t)(b * 1.1) + (1u << 20);
}

struct Request {
    unsigned long long id;
    bura_request r;
    PlanClass cls;
    Clock::time_point t_submit, t_start, t_end;
    bool done = false;
    bura_request_info info{};
};

struct Resident {
    PlanClass cls;
    bura_plan* plan = nullptr;  // null while a worker sets it up
    size_t bytes = 0;
    bool busy = false;
    double alpha = 0.0;
    unsigned long long last_use = 0;
};

}  // namespace

struct bura_server {
    bura_server_options opt{};
    int dev = 0;
    std::mutex m;
    std::condition_variable cv_work;  // queue non-empty or stopping
    std::condition_variable cv_done;  // a request finished
    std::condition_variable cv_pool;  // a plan became idle or was freed
    std::deque<Request*> queue;
    std::unordered_map<unsigned long long, Request*> reqs;
    std::vector<Resident*> pool;
    std::vector<std::pair<PlanClass, size_t>> class_bytes;  // measured plan sizes per class
    size_t resident_bytes = 0;
    unsigned long long next_id = 1, tick = 0;
    bool stop = false;
    bura_server_stats st{};
    std::vector<std::thread> workers;

    size_t bytes_for(const bura_request& r) {
        const PlanClass c = class_of(r);
        for (auto& e : class_bytes)
            if (e.first == c) return e.second;
        return estimate_bytes(r, opt.plan);
    }

    // Under the lock: an idle resident plan of the class (preferring one already at alpha), or a new
    // slot reserved for a plan to set up, or null when the request must wait.  Evicted plans are
    // handed back in `evict` to be destroyed outside the lock.
    Resident* acquire(const Request& q, std::vector<Resident*>& evict) {
        Resident* best = nullptr;
        for (Resident* e : pool)
            if (!e->busy && e->plan && e->cls == q.cls && (!best || e->alpha == q.r.alpha)) best = e;
        if (best) {
            best->busy = true;
            return best;
        }
        const size_t need = bytes_for(q.r);
        bool any_busy = false;
        for (Resident* e : pool) any_busy = any_busy || e->busy;
        while (resident_bytes + need > opt.mem_budget) {
            Resident* lru = nullptr;
            for (Resident* e : pool)
                if (!e->busy && (!lru || e->last_use < lru->last_use)) lru = e;
            if (!lru) break;
            pool.erase(std::find(pool.begin(), pool.end(), lru));
            resident_bytes -= lru->bytes;
            st.evictions += 1;
            evict.push_back(lru);
        }
        if (resident_bytes + need > opt.mem_budget && any_busy) return nullptr;  // wait for a plan to go idle
        Resident* e = new Resident();
        e->cls = q.cls;
        e->busy = true;
        e->bytes = need;
        resident_bytes += need;
        pool.push_back(e);
        return e;
    }

    void serve(Request* q, cudaStream_t s) {
        std::vector<Resident*> evict;
        Resident* e = nullptr;
        {
            std::unique_lock<std::mutex> lk(m);
            while (!(e = acquire(*q, evict))) {
                lk.unlock();
                for (Resident* v : evict) { bura_destroy(v->plan); delete v; }
                evict.clear();
                lk.lock();
                if ((e = acquire(*q, evict))) break;
                cv_pool.wait(lk);
            }
        }
        for (Resident* v : evict) { bura_destroy(v->plan); delete v; }
        bura_request_info& info = q->info;
        int rc = BURA_OK;
        if (!e->plan) {
            bura_plan* p = nullptr;
            rc = bura_setup(&q->r.grid, q->r.faces, q->r.alpha, q->r.k, &opt.plan, &p);
            std::lock_guard<std::mutex> lk(m);
            if (rc == BURA_OK) {
                bura_stats ps;
                bura_get_stats(p, &ps);
                resident_bytes = resident_bytes - e->bytes + ps.device_bytes;
                e->bytes = ps.device_bytes;
                bool known = false;
                for (auto& cb : class_bytes)
                    if (cb.first == e->cls) { cb.second = ps.device_bytes; known = true; }
                if (!known) class_bytes.push_back({e->cls, ps.device_bytes});
                e->plan = p;
                e->alpha = q->r.alpha;
                st.builds += 1;
                info.built = 1;
            } else {  // give the slot back
                pool.erase(std::find(pool.begin(), pool.end(), e));
                resident_bytes -= e->bytes;
                delete e;
                e = nullptr;
                cv_pool.notify_all();
            }
        } else if (e->alpha != q->r.alpha) {
            rc = bura_retarget(e->plan, q->r.alpha);
            std::lock_guard<std::mutex> lk(m);
            if (rc == BURA_OK) {
                e->alpha = q->r.alpha;
                st.retargets += 1;
                info.retargeted = 1;
            }
        } else {
            std::lock_guard<std::mutex> lk(m);
            st.reuses += 1;
        }
        if (e && rc == BURA_OK) {
            rc = bura_solve_host(e->plan, q->r.f, q->r.u, q->r.tol, s);
            bura_stats ps;
            if (bura_get_stats(e->plan, &ps) == BURA_OK) {
                info.iters = ps.iters;
                info.outer = ps.outer;
                info.err_bound = ps.err_bound;
            }
        }
        std::lock_guard<std::mutex> lk(m);
        if (e) {
            e->busy = false;
            e->last_use = ++tick;
            if (rc != BURA_OK && rc != BURA_ENOCONV && e->plan) {  // a plan in an unknown state is not reused
                pool.erase(std::find(pool.begin(), pool.end(), e));
                resident_bytes -= e->bytes;
                bura_destroy(e->plan);
                delete e;
            }
            cv_pool.notify_all();
        }
        q->t_end = Clock::now();
        info.status = rc;
        info.queue_ms = ms_between(q->t_submit, q->t_start);
        info.service_ms = ms_between(q->t_start, q->t_end);
        info.total_ms = ms_between(q->t_submit, q->t_end);
        q->done = true;
        st.completed += 1;
        cv_done.notify_all();
    }

    void worker() {
        cudaSetDevice(dev);
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) s = nullptr;
        for (;;) {
            Request* q = nullptr;
            {
                std::unique_lock<std::mutex> lk(m);
                cv_work.wait(lk, [&] { return stop || !queue.empty(); });
                if (queue.empty()) break;  // stopping and drained
                q = queue.front();
                queue.pop_front();
                q->t_start = Clock::now();
            }
            if (!s) {  // no stream: fail the request rather than run on the legacy stream
                std::lock_guard<std::mutex> lk(m);
                q->t_end = Clock::now();
                q->info.status = BURA_ECUDA;
                q->info.total_ms = ms_between(q->t_submit, q->t_end);
                q->done = true;
                st.completed += 1;
                cv_done.notify_all();
                continue;
            }
            serve(q, s);
        }
        if (s) {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
    }
};

extern "C" {

void bura_server_default_options(bura_server_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->workers = 8;
    o->mem_budget = 0;
    bura_default_options(&o->plan);
}

int bura_server_create(const bura_server_options* opt, bura_server** out) {
    if (!out) return BURA_EINVAL;
    *out = nullptr;
    bura_server_options o;
    bura_server_default_options(&o);
    if (opt) o = *opt;
    if (o.workers < 0 || o.workers > 256) return BURA_EINVAL;
    if (o.workers == 0) o.workers = 8;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BURA_ECUDA;
    if (o.mem_budget == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return BURA_ECUDA;
        o.mem_budget = (size_t)(0.8 * (double)fr);
    }
    bura_server* srv = new (std::nothrow) bura_server();
    if (!srv) return BURA_ENOMEM;
    srv->opt = o;
    srv->dev = dev;
    srv->st.mem_budget = o.mem_budget;
    srv->workers.reserve(o.workers);
    for (int w = 0; w < o.workers; ++w) srv->workers.emplace_back([srv] { srv->worker(); });
    *out = srv;
    return BURA_OK;
}

int bura_server_submit(bura_server* srv, const bura_request* req, unsigned long long* id) {
    if (!srv || !req || !id || !req->f || !req->u) return BURA_EINVAL;
    const bura_grid& g = req->grid;
    if (g.dim != 2 && g.dim != 3) return BURA_EINVAL;
    for (int a = 0; a < g.dim; ++a)
        if (g.n[a] < 1) return BURA_EINVAL;
    if (g.coef_kind != BURA_COEF_CONSTANT && (g.coef_kind != BURA_COEF_FACES || !req->faces)) return BURA_EINVAL;
    if (!(req->alpha > 0 && req->alpha < 1) || req->k < 1 || req->k > BURA_MAX_K || !(req->tol > 0)) return BURA_EINVAL;
    Request* q = new (std::nothrow) Request();
    if (!q) return BURA_ENOMEM;
    q->r = *req;
    q->cls = class_of(*req);
    q->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(srv->m);
        if (srv->stop) {
            delete q;
            return BURA_EINVAL;
        }
        q->id = srv->next_id++;
        srv->reqs[q->id] = q;
        srv->queue.push_back(q);
        srv->st.submitted += 1;
        *id = q->id;
    }
    srv->cv_work.notify_one();
    return BURA_OK;
}

int bura_server_wait(bura_server* srv, unsigned long long id, double timeout_s, bura_request_info* info) {
    if (!srv) return BURA_EINVAL;
    std::unique_lock<std::mutex> lk(srv->m);
    auto it = srv->reqs.find(id);
    if (it == srv->reqs.end()) return BURA_EINVAL;
    Request* q = it->second;
    if (timeout_s < 0) srv->cv_done.wait(lk, [&] { return q->done; });
    else if (!srv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return q->done; }))
        return BURA_ETIMEOUT;
    if (info) *info = q->info;
    srv->reqs.erase(id);
    delete q;
    return BURA_OK;
}

int bura_server_get_stats(bura_server* srv, bura_server_stats* out) {
    if (!srv || !out) return BURA_EINVAL;
    std::lock_guard<std::mutex> lk(srv->m);
    *out = srv->st;
    out->resident_plans = (int)srv->pool.size();
    out->resident_bytes = srv->resident_bytes;
    return BURA_OK;
}

int bura_server_destroy(bura_server* srv) {
    if (!srv) return BURA_OK;
    {
        std::lock_guard<std::mutex> lk(srv->m);
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    for (auto& t : srv->workers) t.join();
    cudaSetDevice(srv->dev);
    for (Resident* e : srv->pool) {
        bura_destroy(e->plan);
        delete e;
    }
    for (auto& kv : srv->reqs) delete kv.second;
    delete srv;
    return BURA_OK;
}

}  // extern "C"
