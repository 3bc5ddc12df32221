// cp_server: rectangle solves of mixed lattice / L / N / primes served with
// continuous batching.
//
// Requests are solved as jobs: one strip (Sec. 3, eq. (Z_from_T)) at full
// degree D = L N - 1.  At admission, queued requests for the same rectangle
// (lattice, L, N) are merged into one job whose vector rows carry all their
// primes (padded to a multiple of four with repeats of the last prime, so that
// rows are 16-byte chunked); they share the job's tables, launches and index
// traffic.  A job's vectors live in a device arena owned by the server (one
// allocation made at creation, so admission never calls cudaMalloc); its
// tables come from the per-device cache.  A step issues ONE batched gather
// launch (two if some rows cannot take the TMA kernel) holding the next
// per-site factor of every active job: row factors T_i while the strip grows,
// then its read-out chain T_i^last, then the extraction of the e_0 row.
// Requests that arrive while others run are admitted at the next step if
// their job's footprint fits the free arena (first fit, queue order; a job
// that does not fit yet does not block smaller ones); finished jobs return
// their memory at once.
#include <cuda_runtime.h>

#include <chrono>
#include <deque>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "cp_internal.h"

using namespace cp;

namespace {

// First-fit allocator over one device allocation.
struct Arena {
    char *base = nullptr;
    size_t size = 0;
    std::map<size_t, size_t> free_;  // offset -> bytes

    int init(size_t bytes) {
        size = bytes;
        int rc = dev_alloc((void **)&base, bytes);
        if (rc) return rc;
        free_[0] = bytes;
        return CP_OK;
    }
    bool alloc(size_t bytes, size_t *off) {
        bytes = (bytes + 255) & ~(size_t)255;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            size_t rest = it->second - bytes;
            size_t at = it->first + bytes;
            free_.erase(it);
            if (rest) free_[at] = rest;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + 255) & ~(size_t)255;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t largest() const {
        size_t m = 0;
        for (auto &f : free_) m = std::max(m, f.second);
        return m;
    }
    size_t free_bytes() const {
        size_t s = 0;
        for (auto &f : free_) s += f.second;
        return s;
    }
    ~Arena() { dev_free(base); }
};

enum ReqState { REQ_QUEUED = 0, REQ_ACTIVE = 1, REQ_DONE = 2, REQ_FAILED = -1 };

struct Request {
    uint64_t id = 0;
    int lattice = 0, L = 0, N = 0, P = 0;
    std::vector<uint32_t> primes;
    int state = REQ_QUEUED;
    std::vector<uint32_t> result;  // [P][L*N]
    double t_submit = 0, t_admit = 0, t_done = 0;
};

struct Job {
    int lattice = 0, L = 0, N = 0, P = 0, D1 = 0;  // P: padded prime count
    std::vector<uint32_t> primes;                  // padded
    std::vector<std::pair<Request *, int>> members;  // request, first prime index in the row
    std::shared_ptr<TableSet> tabs;
    size_t off = 0, bytes = 0;  // arena block
    uint32_t *vec[2] = {nullptr, nullptr}, *scratch[2] = {nullptr, nullptr}, *row = nullptr, *tr = nullptr;
    uint32_t *primes_dev = nullptr;
    int op = 0, n_ops = 0;  // next factor, number of factors (rows + read-out)
    std::vector<uint32_t> result;  // [P][D1]
};

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct cp_server {
    Arena arena;
    cudaStream_t stream = nullptr;
    int max_active = 0;
    uint64_t next_id = 1;
    std::deque<Request *> queue;
    std::vector<std::unique_ptr<Job>> active;
    std::map<uint64_t, std::unique_ptr<Request>> reqs;
    GatherTask *tasks_dev = nullptr;
    size_t tasks_cap = 0;
    std::vector<uint64_t> finished;  // ids finished since the last poll
    uint64_t steps = 0, launches = 0, updates = 0;
    ~cp_server() {
        if (stream) cudaStreamSynchronize(stream);
        dev_free(tasks_dev);
    }
};

static size_t request_bytes(const TableSet &ts, int L, size_t RB) {
    (void)L;
    const uint64_t sA = ts.last[0].n_dst, sB = ts.last.size() >= 2 ? ts.last[1].n_dst : 1;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    return 2 * al(ts.S_max * RB) + al(sA * RB) + al(sB * RB) + 2 * al(RB) + al(4 * CP_MAX_PRIMES);
}

// Motzkin numbers M_0..M_{CP_MAX_L+1} by eq. (M_recurs), for footprints.
struct MotzkinTable {
    uint64_t M[CP_MAX_L + 2];
    MotzkinTable() {
        M[0] = M[1] = 1;
        for (int p = 2; p <= CP_MAX_L + 1; ++p) {
            M[p] = M[p - 1];
            for (int k = 0; k <= p - 2; ++k) M[p] += M[k] * M[p - k - 2];
        }
    }
};
static const MotzkinTable g_motzkin;

// Footprint of a job without building its tables.
static size_t request_bytes_estimate(int lattice, int L, int D1, int P) {
    const uint64_t *M = g_motzkin.M;
    auto cnt = [&](int n) -> uint64_t { return n == 0 ? 1 : M[n - 1]; };
    const size_t RB = (size_t)D1 * P * 4;
    const uint64_t Smax = (lattice == CP_SQUARE && L >= 2) ? cnt(L) + cnt(L - 1) : cnt(L);
    const uint64_t sA = L >= 2 ? cnt(L - 1) : 1, sB = L >= 3 ? cnt(L - 2) : 1;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    return 2 * al(Smax * RB) + al(sA * RB) + al(sB * RB) + 2 * al(RB) + al(4 * CP_MAX_PRIMES);
}

// Largest padded prime count of a job on D1 coefficients: the row must stay a
// TMA row (at most 1536 16-byte chunks) and within CP_MAX_PRIMES.
static int job_prime_limit(int D1) {
    int lim = (6144 / D1) & ~3;
    if (lim > CP_MAX_PRIMES) lim = CP_MAX_PRIMES;
    return lim < 4 ? 4 : lim;
}

static int admit(cp_server *sv, Job *j, bool *fits) {
    *fits = false;
    int rc;
    if (!j->tabs && (rc = get_tables(j->lattice, j->L, (size_t)j->D1 * j->P * 4, sv->stream, &j->tabs))) return rc;
    const TableSet &ts = *j->tabs;
    const size_t RB = (size_t)j->D1 * j->P * 4;
    j->bytes = request_bytes(ts, j->L, RB);
    size_t off = 0;
    if (!sv->arena.alloc(j->bytes, &off)) return CP_OK;
    *fits = true;
    j->off = off;
    char *p = sv->arena.base + off;
    auto take = [&](size_t b) {
        char *q = p;
        p += (b + 255) & ~(size_t)255;
        return reinterpret_cast<uint32_t *>(q);
    };
    const uint64_t sA = ts.last[0].n_dst, sB = ts.last.size() >= 2 ? ts.last[1].n_dst : 1;
    j->vec[0] = take(ts.S_max * RB);
    j->vec[1] = take(ts.S_max * RB);
    j->scratch[0] = take(sA * RB);
    j->scratch[1] = take(sB * RB);
    j->row = take(RB);
    j->tr = take(RB);
    j->primes_dev = take(4 * CP_MAX_PRIMES);
    CP_CUDA_TRY(cudaMemcpyAsync(j->primes_dev, j->primes.data(), 4 * j->P, cudaMemcpyHostToDevice, sv->stream));
    CP_CUDA_TRY(cudaMemsetAsync(j->vec[0], 0, ts.S_b * RB, sv->stream));
    static const uint32_t ones[CP_MAX_PRIMES] = {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1,
                                                 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1};
    CP_CUDA_TRY(cudaMemcpyAsync(j->vec[0], ones, 4 * j->P, cudaMemcpyHostToDevice, sv->stream));
    j->op = 0;
    j->n_ops = (j->N - 1) * (int)ts.row.size() + (int)ts.last.size();
    return CP_OK;
}

// Task of job j's next factor; returns true if this was the last one.
static bool next_tasks(Job *j, std::vector<GatherTask> *tasks, uint64_t *upd) {
    const TableSet &ts = *j->tabs;
    const int nrow = (int)ts.row.size();
    const int main_ops = (j->N - 1) * nrow;
    const SiteTable *tab;
    const uint32_t *in;
    uint32_t *out;
    bool partial = true;  // every output but the result feeds further gathers only
    if (j->op < main_ops) {
        const int i = j->op % nrow;
        tab = &ts.row[i];
        in = j->vec[j->op & 1];
        out = j->vec[(j->op & 1) ^ 1];
    } else {
        const int k = j->op - main_ops;
        tab = &ts.last[k];
        in = k == 0 ? j->vec[main_ops & 1] : j->scratch[(k - 1) & 1];
        partial = k + 1 < (int)ts.last.size();
        out = partial ? j->scratch[k & 1] : j->row;
    }
    append_gather_tasks(tasks, *tab, in, out, j->primes_dev, j->D1, j->P, partial);
    // updates count the requested primes only (padding lanes are not work asked for)
    int real = 0;
    for (auto &m : j->members) real += m.first->P;
    *upd += tab->n_site_out * (uint64_t)j->D1 * real;
    return ++j->op == j->n_ops;
}

static int launch_batch(cp_server *sv, std::vector<GatherTask> &tasks) {
    if (tasks.empty()) return CP_OK;
    // TMA-able tasks in one launch, the others in a register-kernel launch
    std::vector<GatherTask> a, b;
    for (auto &t : tasks) (tma_usable(t) ? a : b).push_back(t);
    std::vector<GatherTask> all;
    int tile_a = 0, tile_b = kGatherItems;
    uint32_t blk_a = 0, blk_b = 0;
    if (!a.empty()) {
        tile_a = effective_tile(a, make_tile(default_rows(a), 0, 0, 0));
        blk_a = assign_blocks(a, tile_a);
    }
    if (!b.empty()) blk_b = assign_blocks(b, tile_b);
    all.insert(all.end(), a.begin(), a.end());
    all.insert(all.end(), b.begin(), b.end());
    if (all.size() > sv->tasks_cap) {
        dev_free(sv->tasks_dev);
        sv->tasks_dev = nullptr;
        size_t cap = std::max<size_t>(64, all.size() * 2);
        int rc = dev_alloc((void **)&sv->tasks_dev, cap * sizeof(GatherTask));
        if (rc) return rc;
        sv->tasks_cap = cap;
    }
    CP_CUDA_TRY(cudaMemcpyAsync(sv->tasks_dev, all.data(), all.size() * sizeof(GatherTask), cudaMemcpyHostToDevice,
                                sv->stream));
    int rc;
    if (!a.empty() && (rc = launch_gather(sv->tasks_dev, (int)a.size(), blk_a, tile_a, sv->stream))) return rc;
    if (!b.empty() && (rc = launch_gather(sv->tasks_dev + a.size(), (int)b.size(), blk_b, tile_b, sv->stream)))
        return rc;
    sv->launches += (a.empty() ? 0 : 1) + (b.empty() ? 0 : 1);
    return CP_OK;
}

extern "C" int cp_server_create(size_t mem_budget_bytes, int max_active, void *cuda_stream, cp_server **out) {
    if (!out) return fail(CP_EINVAL, "out is NULL");
    *out = nullptr;
    if (mem_budget_bytes < (1u << 20)) return fail(CP_EINVAL, "memory budget below 1 MiB");
    if (max_active < 1) return fail(CP_EINVAL, "max_active must be >= 1");
    auto sv = std::make_unique<cp_server>();
    sv->stream = (cudaStream_t)cuda_stream;
    sv->max_active = max_active;
    int rc;
    if ((rc = prepare_gather_kernels()) || (rc = crt_static_touch())) return rc;
    if ((rc = sv->arena.init(mem_budget_bytes))) return rc;
    *out = sv.release();
    return CP_OK;
}

extern "C" int cp_server_submit(cp_server *sv, int lattice, int L, int N, const uint32_t *primes, int n_primes,
                                uint64_t *req_id) {
    if (!sv || !req_id) return fail(CP_EINVAL, "NULL argument");
    if (lattice != CP_SQUARE && lattice != CP_TRIANGULAR) return fail(CP_EINVAL, "bad lattice");
    if (L < 1 || L > CP_MAX_L || N < 1 || (long long)L * N > (1 << 16)) return fail(CP_EINVAL, "bad L or N");
    int rc = check_primes(primes, n_primes);
    if (rc) return rc;
    auto r = std::make_unique<Request>();
    r->id = sv->next_id++;
    r->lattice = lattice;
    r->L = L;
    r->N = N;
    r->P = n_primes;
    r->primes.assign(primes, primes + n_primes);
    r->t_submit = now_s();
    if (request_bytes_estimate(lattice, L, L * N, (n_primes + 3) & ~3) > sv->arena.size)
        return fail(CP_ENOMEM, "request footprint exceeds the server's memory budget");
    *req_id = r->id;
    sv->queue.push_back(r.get());
    sv->reqs[r->id] = std::move(r);
    return CP_OK;
}

// One step: admit what fits, one batched launch of the next factor of every
// active job, extract and retire the finished ones.  Synchronous.
extern "C" int cp_server_step(cp_server *sv, int *n_active, int *n_queued, int *n_finished) {
    if (!sv) return fail(CP_EINVAL, "server is NULL");
    int rc;
    // admission: rectangles in the queue order of their first request; queued
    // requests of the same rectangle form one job (merged while the row stays a
    // TMA row and the job fits the largest free block)
    std::vector<Request *> q(sv->queue.begin(), sv->queue.end());
    std::vector<char> taken(q.size(), 0);
    std::map<uint64_t, std::vector<size_t>> by_shape;
    std::vector<uint64_t> order;
    for (size_t a = 0; a < q.size(); ++a) {
        const uint64_t key = ((uint64_t)q[a]->lattice << 40) | ((uint64_t)q[a]->L << 20) | (uint64_t)q[a]->N;
        auto &v = by_shape[key];
        if (v.empty()) order.push_back(key);
        v.push_back(a);
    }
    for (uint64_t key : order) {
        auto &members = by_shape[key];
        size_t next = 0;
        while (next < members.size() && (int)sv->active.size() < sv->max_active) {
            Request *r = q[members[next]];
            auto job = std::make_unique<Job>();
            job->lattice = r->lattice;
            job->L = r->L;
            job->N = r->N;
            job->D1 = r->L * r->N;
            const int lim = job_prime_limit(job->D1);
            const size_t room = sv->arena.largest();
            std::vector<size_t> picked;
            int P = 0;
            size_t b = next;
            for (; b < members.size(); ++b) {
                Request *o = q[members[b]];
                if (!picked.empty() && (P + o->P > lim || request_bytes_estimate(r->lattice, r->L, job->D1,
                                                                                 (P + o->P + 3) & ~3) > room))
                    break;
                picked.push_back(members[b]);
                job->members.push_back({o, P});
                job->primes.insert(job->primes.end(), o->primes.begin(), o->primes.end());
                P += o->P;
            }
            while (job->primes.size() % 4) job->primes.push_back(job->primes.back());  // padding lanes
            job->P = (int)job->primes.size();
            bool fits = false;
            if ((rc = admit(sv, job.get(), &fits))) return rc;
            if (!fits) break;  // this rectangle waits; smaller ones may still fit
            const double t = now_s();
            for (size_t idx : picked) {
                taken[idx] = 1;
                q[idx]->state = REQ_ACTIVE;
                q[idx]->t_admit = t;
            }
            sv->active.push_back(std::move(job));
            next = b;
        }
        if ((int)sv->active.size() >= sv->max_active) break;
    }
    sv->queue.clear();
    for (size_t a = 0; a < q.size(); ++a)
        if (!taken[a]) sv->queue.push_back(q[a]);
    // one batched launch of every active job's next factor
    std::vector<GatherTask> tasks;
    std::vector<Job *> finishing;
    uint64_t upd = 0;
    for (auto &j : sv->active)
        if (next_tasks(j.get(), &tasks, &upd)) finishing.push_back(j.get());
    if ((rc = launch_batch(sv, tasks))) return rc;
    for (Job *j : finishing) {
        if ((rc = launch_transpose_row(j->row, j->tr, j->D1, j->P, sv->stream))) return rc;
        j->result.resize((size_t)j->P * j->D1);
        CP_CUDA_TRY(cudaMemcpyAsync(j->result.data(), j->tr, 4ull * j->P * j->D1, cudaMemcpyDeviceToHost, sv->stream));
    }
    if ((rc = check_device_error(sv->stream))) return rc;  // synchronises the stream
    const double t = now_s();
    int n_req_done = 0;
    for (Job *j : finishing) {
        for (auto &m : j->members) {
            Request *r = m.first;
            r->result.assign(j->result.begin() + (size_t)m.second * j->D1,
                             j->result.begin() + (size_t)(m.second + r->P) * j->D1);
            r->state = REQ_DONE;
            r->t_done = t;
            sv->finished.push_back(r->id);
            ++n_req_done;
        }
        sv->arena.release(j->off, j->bytes);
    }
    for (size_t k = 0; k < sv->active.size();) {
        if (sv->active[k]->op == sv->active[k]->n_ops) sv->active.erase(sv->active.begin() + k);
        else ++k;
    }
    sv->steps++;
    sv->updates += upd;
    if (n_active) {
        int na = 0;
        for (auto &j : sv->active) na += (int)j->members.size();
        *n_active = na;
    }
    if (n_queued) *n_queued = (int)sv->queue.size();
    if (n_finished) *n_finished = n_req_done;
    return CP_OK;
}

extern "C" int cp_server_result(cp_server *sv, uint64_t req_id, uint32_t *out_host, size_t out_len, int *state,
                                double times_s[3]) {
    if (!sv || !state) return fail(CP_EINVAL, "NULL argument");
    auto it = sv->reqs.find(req_id);
    if (it == sv->reqs.end()) return fail(CP_EINVAL, "unknown request id");
    Request *r = it->second.get();
    *state = r->state;
    if (times_s) {
        times_s[0] = r->t_submit;
        times_s[1] = r->t_admit;
        times_s[2] = r->t_done;
    }
    if (r->state != REQ_DONE || !out_host) return CP_OK;
    if (out_len < r->result.size()) return fail(CP_EINVAL, "out_len < n_primes * L * N");
    std::copy(r->result.begin(), r->result.end(), out_host);
    return CP_OK;
}

extern "C" int cp_server_cancel(cp_server *sv, uint64_t req_id) {
    if (!sv) return fail(CP_EINVAL, "server is NULL");
    auto it = sv->reqs.find(req_id);
    if (it == sv->reqs.end()) return fail(CP_EINVAL, "unknown request id");
    Request *r = it->second.get();
    if (r->state != REQ_QUEUED) return fail(CP_EINVAL, "only a queued request can be cancelled");
    for (auto q = sv->queue.begin(); q != sv->queue.end(); ++q)
        if (*q == r) {
            sv->queue.erase(q);
            break;
        }
    r->state = REQ_FAILED;
    return CP_OK;
}

extern "C" int cp_server_poll(cp_server *sv, uint64_t *ids_out, int max_ids, int *n_ids) {
    if (!sv || !n_ids || (max_ids > 0 && !ids_out)) return fail(CP_EINVAL, "bad arguments");
    const int n = (int)std::min<size_t>((size_t)std::max(max_ids, 0), sv->finished.size());
    for (int k = 0; k < n; ++k) ids_out[k] = sv->finished[k];
    sv->finished.erase(sv->finished.begin(), sv->finished.begin() + n);
    *n_ids = n;
    return CP_OK;
}

extern "C" int cp_server_release(cp_server *sv, uint64_t req_id) {
    if (!sv) return fail(CP_EINVAL, "server is NULL");
    auto it = sv->reqs.find(req_id);
    if (it == sv->reqs.end()) return fail(CP_EINVAL, "unknown request id");
    if (it->second->state == REQ_ACTIVE || it->second->state == REQ_QUEUED)
        return fail(CP_EINVAL, "request still in flight");
    sv->reqs.erase(it);
    return CP_OK;
}

extern "C" int cp_server_stats(const cp_server *sv, uint64_t *steps, uint64_t *launches, uint64_t *updates,
                               size_t *arena_free_bytes) {
    if (!sv) return fail(CP_EINVAL, "server is NULL");
    if (steps) *steps = sv->steps;
    if (launches) *launches = sv->launches;
    if (updates) *updates = sv->updates;
    if (arena_free_bytes) *arena_free_bytes = sv->arena.free_bytes();
    return CP_OK;
}

extern "C" void cp_server_destroy(cp_server *sv) { delete sv; }
