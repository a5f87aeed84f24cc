// Serving: threshold-point queries (Algorithm 1, Sec. 3.3) over several
// resident instances with continuous batching.
//
// Every query is an Algorithm 1 state machine on the host.  Two ways to
// batch the supporting points the queries wait for:
//
//  * across instances (merge_instances = 1): instances are
//    grouped by their arithmetic (precision path and stopping rules, so a
//    result is the one the instance gives alone) and by size (a round lasts
//    as long as its slowest pair); each group has one context holding its
//    instances' products (a pair list) and its own round thread and stream,
//    and one device round takes the waiting queries of every instance of
//    the group (up to max_batch) as the columns of one batch of weight
//    vectors.  Query k's column weighs only its instance's agents and
//    tasks, so every other product starts that column frozen at value 0 and
//    costs nothing.  After the round the host takes each query's assignment
//    on its instance's block of c, one Algorithm 4 call evaluates every
//    query's assigned pairs, and the Algorithm 1 steps run on the worker
//    threads while the next round is already on the device.
//  * per instance (merge_instances = 0, the default): an idle instance takes its own
//    waiting queries as one morap_supporting_points batch on its own
//    stream; the batches of different instances overlap on the device.
//
// A round of the merged mode sweeps every weight column of every product it
// touches (the [state][weight] layout computes a product's columns
// together), so a round over many instances does the work of each product
// once per column of the round: it lowers latency at light load and lowers
// the saturation throughput; per-instance batches keep every column of a
// round useful.
//
// Queries that arrive while a round runs join the next one.  Queries are
// admitted in arrival order while the device bytes their weights occupy
// (values, recorded actions, schedulers) fit the budget; results do not
// depend on the batch a query rides in, because each (product, weight) pair
// runs exactly its own sweeps.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace morap {

}  // namespace morap

using namespace morap;

struct ServerQuery {
    int64_t ticket;
    int inst;
    Alg1 ps;
    std::chrono::steady_clock::time_point t_submit, t_done;
    bool admitted = false;
    int64_t cost = 0;
};

struct morap_server {
    std::vector<morap_ctx *> inst;
    std::vector<int> n_obj, n_tasks;
    std::vector<int64_t> bytes_per_weight;
    std::vector<cudaStream_t> streams;
    std::vector<char> busy;
    morap_server_config cfg{};
    std::mutex mu;
    std::condition_variable cv, cv_done;
    std::deque<int64_t> pending;                 // submitted, not admitted (arrival order)
    std::vector<std::deque<int64_t>> ready;      // admitted, waiting for a supporting point
    std::unordered_map<int64_t, ServerQuery> queries;
    int64_t next_ticket = 1, in_use = 0;
    bool stop = false;
    std::vector<std::thread> workers;
    std::thread scheduler;
    std::deque<int> jobs;  // instances with a batch to run
    // merged mode: instances are grouped by arithmetic (the same results as
    // alone) and by size (a round lasts as long as its slowest pair); each
    // group has one context holding its instances' products, its own stream,
    // ready queue and round thread
    struct Group {
        morap_ctx *merged = nullptr;
        cudaStream_t stream = nullptr;
        std::vector<int> members;                  // instance indices
        std::vector<int32_t> agent_off, task_off, pair_off;  // per member
        int n_agents_total = 0, n_obj_total = 0, n_products = 0;
        std::deque<int64_t> ready;                 // admitted queries waiting for a supporting point
        std::thread thread;
    };
    std::vector<Group> groups;
    std::vector<int> group_of, member_of;          // per instance
    std::vector<int32_t> n_agents;
    bool merged = false;
    struct StepJob {
        int64_t ticket;
        std::vector<double> r;
        std::vector<int32_t> f;
        int status;
    };
    std::deque<StepJob> steps;      // Algorithm 1 steps for the worker threads
    // stats
    std::vector<double> latencies_ms;
    int64_t submitted = 0, completed = 0, batches = 0, batch_queries = 0;
    std::chrono::steady_clock::time_point t_first{}, t_last{};
    bool have_first = false;
};

namespace {

void scheduler_loop(morap_server *S) {
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stop) {
        // admission in arrival order, by the device bytes of one weight slot
        bool admitted = false;
        while (!S->pending.empty()) {
            ServerQuery &q = S->queries[S->pending.front()];
            if (S->cfg.hbm_budget && S->in_use + q.cost > (int64_t)S->cfg.hbm_budget && S->in_use > 0) break;
            q.admitted = true;
            S->in_use += q.cost;
            if (S->merged)
                S->groups[S->group_of[q.inst]].ready.push_back(q.ticket);
            else
                S->ready[q.inst].push_back(q.ticket);
            S->pending.pop_front();
            admitted = true;
        }
        bool dispatched = S->merged && admitted;  // the groups' round threads wait for admitted queries
        for (size_t i = 0; i < S->inst.size() && !S->merged; ++i)
            if (!S->busy[i] && !S->ready[i].empty()) {
                S->busy[i] = 1;
                S->jobs.push_back((int)i);
                dispatched = true;
            }
        if (dispatched) S->cv.notify_all();
        S->cv.wait(lk);
    }
}

void worker_loop(morap_server *S) {
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        while (!S->stop && S->jobs.empty()) S->cv.wait(lk);
        if (S->stop) return;
        const int i = S->jobs.front();
        S->jobs.pop_front();
        // take every ready query of the instance (continuous batching)
        std::vector<int64_t> batch;
        while (!S->ready[i].empty() && (int)batch.size() < S->cfg.max_batch) {
            batch.push_back(S->ready[i].front());
            S->ready[i].pop_front();
        }
        const int n = S->n_obj[i];
        const int nJ = S->n_tasks[i];
        std::vector<double> W(batch.size() * n), R(batch.size() * n);
        std::vector<int32_t> F(batch.size() * nJ);
        for (size_t b = 0; b < batch.size(); ++b) {
            const ServerQuery &q = S->queries[batch[b]];
            std::copy(q.ps.w.begin(), q.ps.w.end(), W.begin() + b * n);
        }
        lk.unlock();
        const int rc = morap_supporting_points(S->inst[i], (int32_t)batch.size(), W.data(), (void *)S->streams[i],
                                               R.data(), F.data(), nullptr);
        lk.lock();
        S->batches += 1;
        S->batch_queries += (int64_t)batch.size();
        const auto now = std::chrono::steady_clock::now();
        for (size_t b = 0; b < batch.size(); ++b) {
            ServerQuery &q = S->queries[batch[b]];
            if (rc != MORAP_OK && rc != MORAP_ENOTCONV) {
                q.ps.status = rc;
                q.ps.done = true;
            } else {
                // host QPs of this query, outside the lock, on a private copy
                Alg1 ps = q.ps;
                if (rc == MORAP_ENOTCONV && ps.status == MORAP_OK) ps.status = rc;
                lk.unlock();
                ps.step(R.data() + b * n, F.data() + b * nJ, nJ);
                lk.lock();
                q.ps = std::move(ps);
            }
            if (q.ps.done) {
                q.t_done = now;
                S->in_use -= q.cost;
                S->completed += 1;
                S->latencies_ms.push_back(std::chrono::duration<double, std::milli>(q.t_done - q.t_submit).count());
                S->t_last = now;
            } else {
                S->ready[i].push_back(q.ticket);
            }
        }
        S->busy[i] = 0;
        S->cv.notify_all();
        S->cv_done.notify_all();
    }
}

// Merged mode, device side: one round per batch of waiting queries of any
// instance of group g (Algorithm 3 for every query's weights on the group's
// context, the assignment per query, Algorithm 4 on the assigned pairs of
// all queries in one call); the Algorithm 1 steps go to the worker threads.
void round_loop(morap_server *S, int g) {
    std::unique_lock<std::mutex> lk(S->mu);
    morap_server::Group &G = S->groups[g];
    const int P = G.n_products;
    for (;;) {
        while (!S->stop && G.ready.empty()) S->cv.wait(lk);
        if (S->stop) return;
        std::vector<int64_t> batch;
        while (!G.ready.empty() && (int)batch.size() < S->cfg.max_batch) {
            batch.push_back(G.ready.front());
            G.ready.pop_front();
        }
        const int K = (int)batch.size(), n = G.n_obj_total;
        std::vector<double> W((size_t)K * n, 0.0);
        std::vector<int> inst(K), mem(K);
        for (int k = 0; k < K; ++k) {
            const ServerQuery &q = S->queries[batch[k]];
            const int i = q.inst, m = S->member_of[i], nI = S->n_agents[i], nJ = S->n_tasks[i];
            inst[k] = i;
            mem[k] = m;
            for (int a = 0; a < nI; ++a) W[(size_t)k * n + G.agent_off[m] + a] = q.ps.w[a];
            for (int t = 0; t < nJ; ++t) W[(size_t)k * n + G.n_agents_total + G.task_off[m] + t] = q.ps.w[nI + t];
        }
        lk.unlock();
        std::vector<double> C((size_t)K * P);
        std::vector<int32_t> st((size_t)K * P);
        int rc = morap_solve(G.merged, K, W.data(), (void *)G.stream, C.data(), nullptr, nullptr, st.data());
        std::vector<std::vector<int32_t>> F(K);
        std::vector<int> status(K, MORAP_OK);
        std::vector<int32_t> ev_p, ev_k;
        std::vector<std::pair<int, int>> ev_slot;  // (query, agent) of each evaluated pair
        std::vector<int> ev_task;
        if (rc == MORAP_OK || rc == MORAP_ENOTCONV) {
            for (int k = 0; k < K; ++k) {
                const int i = inst[k], nI = S->n_agents[i], nJ = S->n_tasks[i], p0 = G.pair_off[mem[k]];
                std::vector<double> Ci((size_t)nI * nJ);
                for (int a = 0; a < nI; ++a)
                    for (int t = 0; t < nJ; ++t) {
                        const size_t o = (size_t)k * P + p0 + (size_t)a * nJ + t;
                        Ci[(size_t)a * nJ + t] = C[o];
                        if (st[o] != MORAP_OK) status[k] = MORAP_ENOTCONV;
                    }
                F[k].assign(nJ, -1);
                assign_tasks(nI, nJ, Ci.data(), F[k].data());
                for (int t = 0; t < nJ; ++t)
                    if (F[k][t] >= 0) {
                        ev_p.push_back(p0 + F[k][t] * nJ + t);
                        ev_k.push_back(k);
                        ev_slot.emplace_back(k, F[k][t]);
                        ev_task.push_back(t);
                    }
            }
        }
        std::vector<double> rc_v(ev_p.size()), rp_v(ev_p.size());
        if ((rc == MORAP_OK || rc == MORAP_ENOTCONV) && !ev_p.empty()) {
            const int rc2 = morap_evaluate(G.merged, (int32_t)ev_p.size(), ev_p.data(), ev_k.data(), (void *)G.stream,
                                           rc_v.data(), rp_v.data());
            if (rc2 == MORAP_ENOTCONV) {
                for (auto &sl : ev_slot) status[sl.first] = MORAP_ENOTCONV;
            } else if (rc2 != MORAP_OK) {
                rc = rc2;
            }
        }
        std::vector<morap_server::StepJob> jobs(K);
        for (int k = 0; k < K; ++k) {
            const int i = inst[k], nI = S->n_agents[i], nJ = S->n_tasks[i];
            jobs[k].ticket = batch[k];
            jobs[k].status = (rc == MORAP_OK || rc == MORAP_ENOTCONV) ? status[k] : rc;
            jobs[k].r.assign((size_t)nI + nJ, 0.0);
            jobs[k].f = F[k].empty() ? std::vector<int32_t>(nJ, -1) : F[k];
        }
        for (size_t e = 0; e < ev_p.size(); ++e) {
            const int k = ev_slot[e].first, nI = S->n_agents[inst[k]];
            jobs[k].r[ev_slot[e].second] = rc_v[e];
            jobs[k].r[nI + ev_task[e]] = rp_v[e];
        }
        lk.lock();
        S->batches += 1;
        S->batch_queries += K;
        for (auto &j : jobs) S->steps.push_back(std::move(j));
        S->cv.notify_all();
    }
}

// Merged mode, host side: one Algorithm 1 step per job.
void step_loop(morap_server *S) {
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        while (!S->stop && S->steps.empty()) S->cv.wait(lk);
        if (S->stop) return;
        morap_server::StepJob job = std::move(S->steps.front());
        S->steps.pop_front();
        ServerQuery &q = S->queries[job.ticket];
        if (job.status != MORAP_OK && job.status != MORAP_ENOTCONV) {
            q.ps.status = job.status;
            q.ps.done = true;
        } else {
            Alg1 ps = q.ps;  // host QPs outside the lock, on a private copy
            if (job.status == MORAP_ENOTCONV && ps.status == MORAP_OK) ps.status = job.status;
            lk.unlock();
            ps.step(job.r.data(), job.f.data(), (int)job.f.size());
            lk.lock();
            q.ps = std::move(ps);
        }
        if (q.ps.done) {
            q.t_done = std::chrono::steady_clock::now();
            S->in_use -= q.cost;
            S->completed += 1;
            S->latencies_ms.push_back(std::chrono::duration<double, std::milli>(q.t_done - q.t_submit).count());
            S->t_last = q.t_done;
        } else {
            S->groups[S->group_of[q.inst]].ready.push_back(q.ticket);
        }
        S->cv.notify_all();
        S->cv_done.notify_all();
    }
}

}  // namespace

extern "C" {

void morap_server_config_default(morap_server_config *cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->max_batch = 64;
    cfg->n_workers = 8;
    cfg->eps = 1e-6;
    cfg->max_iter = 64;
    cfg->merge_instances = 0;
}

int morap_server_create(morap_ctx *const *instances, int32_t n_instances, const morap_server_config *cfg_in,
                        morap_server **out) {
    if (!instances || n_instances < 1 || !out) return fail(MORAP_EINVAL, "server: bad arguments");
    morap_server_config cfg;
    if (cfg_in)
        cfg = *cfg_in;
    else
        morap_server_config_default(&cfg);
    if (cfg.max_batch < 1 || cfg.max_batch > 64 || cfg.n_workers < 1 || !(cfg.eps >= 0) || cfg.max_iter < 1 ||
        (cfg.merge_instances != 0 && cfg.merge_instances != 1))
        return fail(MORAP_EINVAL,
                    "server: max_batch in 1..64, n_workers >= 1, eps >= 0, max_iter >= 1, merge_instances 0 or 1");
    auto *S = new morap_server();
    S->cfg = cfg;
    for (int i = 0; i < n_instances; ++i) {
        morap_ctx *c = instances[i];
        int64_t info[10];
        if (!c || morap_product_info(c, 0, info) != MORAP_OK) {
            delete S;
            return fail(MORAP_ESTATE, "server: every instance must be a built context");
        }
        // objectives and device bytes of one weight slot: values (FP32 x2 and
        // double-float x2), recorded action and scheduler per product state
        int64_t states = 0;
        int32_t p = 0;
        int nI = 0, nJ = 0;
        while (morap_product_info(c, p, info) == MORAP_OK) {
            states += info[2];
            nI = std::max<int>(nI, (int)info[8] + 1);
            nJ = std::max<int>(nJ, (int)info[9] + 1);
            ++p;
        }
        set_error("");
        // reserve a full batch up front (when the admission budget allows it),
        // so batches of varying size never allocate or free device memory
        const int64_t bpw = states * (2 * 4 + 2 * 8 + 1 + 1);
        int reserve = cfg.max_batch;
        if (cfg.hbm_budget) reserve = (int)std::min<int64_t>(reserve, std::max<int64_t>(1, (int64_t)cfg.hbm_budget / bpw));
        if (const int rc = ctx_no_tail(c); rc != MORAP_OK) {  // the workers' loops run concurrently
            for (auto s : S->streams) cudaStreamDestroy(s);
            delete S;
            return rc;
        }
        if (ctx_reserve(c, reserve) != MORAP_OK) set_error("");  // not fatal: buffers then grow on demand
        S->inst.push_back(c);
        S->n_obj.push_back(nI + nJ);
        S->n_tasks.push_back(nJ);
        S->n_agents.push_back(nI);
        S->bytes_per_weight.push_back(bpw);
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            for (auto s : S->streams) cudaStreamDestroy(s);
            delete S;
            return fail(MORAP_ECUDA, "server: cudaStreamCreate");
        }
        S->streams.push_back(st);
    }
    S->busy.assign(n_instances, 0);
    S->ready.resize(n_instances);
    if (cfg.merge_instances) {
        // groups: the same arithmetic (so every result is the instance's own)
        // and a similar size (the largest product within a factor of 4)
        std::vector<std::pair<std::string, int>> keys;
        S->group_of.assign(n_instances, -1);
        S->member_of.assign(n_instances, -1);
        for (int i = 0; i < n_instances; ++i) {
            int64_t m = std::max<int64_t>(1, ctx_max_states(instances[i]));
            int bucket = 0;
            while (m > 1) m >>= 2, ++bucket;
            std::pair<std::string, int> key(ctx_arith_key(instances[i]), bucket);
            int g = (int)(std::find(keys.begin(), keys.end(), key) - keys.begin());
            if (g == (int)keys.size()) {
                keys.push_back(key);
                S->groups.emplace_back();
            }
            S->group_of[i] = g;
            S->member_of[i] = (int)S->groups[g].members.size();
            S->groups[g].members.push_back(i);
        }
        int rc = MORAP_OK;
        for (auto &G : S->groups) {
            std::vector<morap_ctx *> cs;
            for (int i : G.members) cs.push_back(instances[i]);
            rc = ctx_merge(cs.data(), (int)cs.size(), &G.merged, G.agent_off, G.task_off, G.pair_off);
            if (rc == MORAP_OK && cudaStreamCreateWithFlags(&G.stream, cudaStreamNonBlocking) != cudaSuccess)
                rc = fail(MORAP_ECUDA, "server: cudaStreamCreate");
            if (rc != MORAP_OK) break;
            const int last = G.members.back();
            G.n_agents_total = G.agent_off.back() + S->n_agents[last];
            G.n_obj_total = G.n_agents_total + G.task_off.back() + S->n_tasks[last];
            G.n_products = G.pair_off.back() + S->n_agents[last] * S->n_tasks[last];
            int64_t bpw = 0;
            for (int i : G.members) bpw += S->bytes_per_weight[i];
            int reserve = cfg.max_batch;
            if (cfg.hbm_budget) reserve = (int)std::min<int64_t>(reserve, std::max<int64_t>(1, (int64_t)cfg.hbm_budget / bpw));
            if ((rc = ctx_no_tail(G.merged)) != MORAP_OK) break;
            if (ctx_reserve(G.merged, reserve) != MORAP_OK) set_error("");  // buffers then grow on demand
        }
        if (rc != MORAP_OK) {
            for (auto &G : S->groups) {
                if (G.merged) morap_ctx_destroy(G.merged);
                if (G.stream) cudaStreamDestroy(G.stream);
            }
            for (auto s : S->streams) cudaStreamDestroy(s);
            delete S;
            return rc;
        }
        S->merged = true;
    }
    S->scheduler = std::thread(scheduler_loop, S);
    if (S->merged) {
        for (size_t g = 0; g < S->groups.size(); ++g) S->groups[g].thread = std::thread(round_loop, S, (int)g);
        for (int k = 0; k < cfg.n_workers; ++k) S->workers.emplace_back(step_loop, S);
    } else {
        for (int k = 0; k < cfg.n_workers; ++k) S->workers.emplace_back(worker_loop, S);
    }
    *out = S;
    return MORAP_OK;
}

int morap_server_destroy(morap_server *S) {
    if (!S) return MORAP_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->scheduler.joinable()) S->scheduler.join();
    for (auto &G : S->groups)
        if (G.thread.joinable()) G.thread.join();
    for (auto &t : S->workers)
        if (t.joinable()) t.join();
    for (auto s : S->streams) cudaStreamDestroy(s);
    for (auto &G : S->groups) {
        if (G.stream) cudaStreamDestroy(G.stream);
        if (G.merged) morap_ctx_destroy(G.merged);
    }
    delete S;
    return MORAP_OK;
}

int morap_submit(morap_server *S, int32_t instance, const double *t, int64_t *ticket_out) {
    if (!S || !t || !ticket_out) return fail(MORAP_EINVAL, "submit: null argument");
    if (instance < 0 || instance >= (int32_t)S->inst.size()) return fail(MORAP_EINVAL, "submit: no such instance");
    const int n = S->n_obj[instance];
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(t[i])) return fail(MORAP_EINVAL, "submit: threshold entries must be finite");
    std::lock_guard<std::mutex> lk(S->mu);
    const int64_t tk = S->next_ticket++;
    ServerQuery &q = S->queries[tk];
    q.ticket = tk;
    q.inst = instance;
    q.ps.init(n, t, nullptr, S->cfg.eps, S->cfg.max_iter);
    q.t_submit = std::chrono::steady_clock::now();
    q.cost = S->bytes_per_weight[instance];
    if (!S->have_first) {
        S->t_first = q.t_submit;
        S->have_first = true;
    }
    S->pending.push_back(tk);
    S->submitted += 1;
    *ticket_out = tk;
    S->cv.notify_all();
    return MORAP_OK;
}

int morap_poll(morap_server *S, int64_t ticket, morap_point_result *res) {
    if (!S || !res) return fail(MORAP_EINVAL, "poll: null argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto itq = S->queries.find(ticket);
    if (itq == S->queries.end()) return fail(MORAP_EINVAL, "poll: unknown ticket");
    const ServerQuery &q = itq->second;
    if (!q.ps.done) return MORAP_EBUSY;
    alg1_result(q.ps, res);
    return MORAP_OK;
}

int morap_server_wait(morap_server *S, double timeout_s) {
    if (!S) return fail(MORAP_EINVAL, "wait: null server");
    std::unique_lock<std::mutex> lk(S->mu);
    const auto until = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    while (S->completed < S->submitted) {
        if (S->cv_done.wait_until(lk, until) == std::cv_status::timeout && S->completed < S->submitted)
            return MORAP_EBUSY;
    }
    return MORAP_OK;
}

int morap_server_stats(morap_server *S, morap_serving_stats *st) {
    if (!S || !st) return fail(MORAP_EINVAL, "stats: null argument");
    std::lock_guard<std::mutex> lk(S->mu);
    std::memset(st, 0, sizeof(*st));
    st->submitted = S->submitted;
    st->completed = S->completed;
    st->batches = S->batches;
    st->mean_batch = S->batches ? (double)S->batch_queries / (double)S->batches : 0.0;
    std::vector<double> l = S->latencies_ms;
    if (!l.empty()) {
        std::sort(l.begin(), l.end());
        auto pct = [&](double q) { return l[std::min(l.size() - 1, (size_t)std::floor(q * (l.size() - 1) + 0.5))]; };
        st->p50_ms = pct(0.50);
        st->p99_ms = pct(0.99);
        const double wall = std::chrono::duration<double>(S->t_last - S->t_first).count();
        st->wall_s = wall;
        st->queries_per_s = wall > 0 ? (double)S->completed / wall : 0.0;
    }
    st->bytes_in_use = S->in_use;
    return MORAP_OK;
}

}  // extern "C"
