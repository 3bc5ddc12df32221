// cp_sweep: the batched finite-lattice sweep (Sec. 4.1-4.3).
//
// For every width r = 1..floor(k/2) one strip is advanced to the largest
// height of the band k-3 <= r+s <= k (s >= r) and read out at every band
// height on the way, so a rectangle shares its strip prefix with the shorter
// ones.  All strips advance in lock-step: global step t applies the t-th
// per-site factor of every strip that still has one, plus the t-th factor of
// any read-out chain in flight, in ONE batched gather launch.  A read-out
// chain T_1^last .. T_{r-1}^last starts at the step where the strip's next
// row begins (both only read the current vector) and runs on two scratch
// buffers while the strip moves on; its last factor writes the e_0 row
// straight into the P~ array.  The primes are split into groups of Pg primes
// (one strip per width and group).  The whole program -- vector resets, every
// batched launch and the series kernel -- is captured once into a CUDA graph,
// so a sweep is a single graph launch.  The gather tile and the prime grouping
// are picked by timing the candidates (autotune) unless given.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "cp_internal.h"
#include "series.h"

using namespace cp;

namespace {

struct SweepStrip {
    int r = 0, group = 0, Pg = 0;
    std::shared_ptr<TableSet> tabs;
    uint32_t *vec[2] = {nullptr, nullptr};
    uint32_t *scratch[2] = {nullptr, nullptr};
    std::vector<int> heights;
};

int n_terms_for(int lattice, int k) {
    if (lattice == CP_SQUARE) return (k % 2 == 1) ? 2 * k - 2 : 2 * k - 3;
    return k;
}

}  // namespace

struct cp_sweep {
    int lattice = 0, k = 0, P = 0, D1 = 0, n = 0, tile = 0, groups = 0, Pg = 0;
    cudaStream_t stream = nullptr;
    uint32_t *primes_dev = nullptr, *ones_dev = nullptr;
    std::vector<SweepStrip> strips;
    std::vector<int2> rects;
    int2 *rects_dev = nullptr;
    uint32_t *ptilde_dev = nullptr;  // [groups][n_rects][D1][Pg]
    uint32_t *series_dev = nullptr;  // [3][P][n]
    uint32_t *crt_dev = nullptr;     // cp_sweep_series_integers: limbs [3][n][limbs], then flags [3][n]
    size_t crt_words = 0;
    std::vector<uint32_t> primes_host;
    int *err_dev = nullptr;
    GatherTask *tasks_dev = nullptr;
    std::vector<uint32_t> step_off, step_ntasks, step_blocks;
    std::vector<int> step_tile;
    uint64_t updates = 0, bytes = 0, site_bytes = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;

    ~cp_sweep() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (auto &s : strips) {
            dev_free(s.vec[0]);
            dev_free(s.vec[1]);
            dev_free(s.scratch[0]);
            dev_free(s.scratch[1]);
        }
        dev_free(primes_dev);
        dev_free(ones_dev);
        dev_free(rects_dev);
        dev_free(ptilde_dev);
        dev_free(series_dev);
        dev_free(crt_dev);
        dev_free(err_dev);
        dev_free(tasks_dev);
    }
};

static int rect_index(const cp_sweep *sw, int r, int s) {
    for (size_t j = 0; j < sw->rects.size(); ++j)
        if (sw->rects[j].x == r && sw->rects[j].y == s) return (int)j;
    return -1;
}

// Accumulate the algorithmic work of one factor: output words, and bytes =
// 4 (S_in + S_out) (D+1) Pg + CSR index bytes.
static void count_work(cp_sweep *sw, const SiteTable &t, int Pg) {
    const uint64_t mid = t.n_site_out - t.n_dst;  // intermediate states of a two-site table (else 0)
    sw->updates += t.n_site_out * (uint64_t)sw->D1 * Pg;
    sw->bytes += 4ull * (t.n_src + t.n_dst) * sw->D1 * Pg + 4ull * (t.n_dst + 1 + t.nnz);
    sw->site_bytes += 4ull * (t.n_src + 2 * mid + t.n_dst) * sw->D1 * Pg + 4ull * (t.n_dst + 1 + t.nnz);
}

// Strips and buffers: one strip per width (and prime group), band rectangles.
static int build_strips(cp_sweep *sw) {
    const int ngroups = sw->groups, Pg = sw->Pg;
    const size_t row_words = (size_t)sw->D1 * Pg;
    int rc;
    // band rectangles (r <= s, k-3 <= r+s <= k), ordered by r then s
    for (int r = 1; 2 * r <= sw->k; ++r)
        for (int s = r; r + s <= sw->k; ++s)
            if (r + s >= sw->k - 3) sw->rects.push_back(make_int2(r, s));
    for (int g = 0; g < ngroups; ++g) {
        for (int r = 1; 2 * r <= sw->k; ++r) {
            SweepStrip st;
            st.r = r;
            st.group = g;
            st.Pg = Pg;
            for (auto &rs : sw->rects)
                if (rs.x == r) st.heights.push_back(rs.y);
            if (st.heights.empty()) continue;
            if ((rc = get_tables(sw->lattice, r, row_words * 4, sw->stream, &st.tabs))) return rc;
            const TableSet &ts = *st.tabs;
            sw->strips.push_back(st);
            SweepStrip &sp = sw->strips.back();
            for (int b = 0; b < 2; ++b)
                if ((rc = dev_alloc((void **)&sp.vec[b], ts.S_max * row_words * 4))) return rc;
            uint64_t sA = ts.last[0].n_dst, sB = ts.last.size() >= 2 ? ts.last[1].n_dst : 1;
            if ((rc = dev_alloc((void **)&sp.scratch[0], sA * row_words * 4))) return rc;
            if ((rc = dev_alloc((void **)&sp.scratch[1], sB * row_words * 4))) return rc;
        }
    }
    return CP_OK;
}

static int enqueue_program(cp_sweep *sw);

// Launch program for gather tile `tile`: per-step task lists, block assignment,
// device task array, and the CUDA graph of the whole sweep.
static int build_program(cp_sweep *sw, int tile) {
    const int Pg = sw->Pg;
    const int n_rects = (int)sw->rects.size();
    const size_t row_words = (size_t)sw->D1 * Pg;
    int rc;
    sw->tile = tile;
    sw->updates = sw->bytes = sw->site_bytes = 0;
    sw->step_off.clear();
    sw->step_ntasks.clear();
    sw->step_blocks.clear();
    sw->step_tile.clear();
    if (sw->exec) cudaGraphExecDestroy(sw->exec);
    if (sw->graph) cudaGraphDestroy(sw->graph);
    sw->exec = nullptr;
    sw->graph = nullptr;
    dev_free(sw->tasks_dev);
    sw->tasks_dev = nullptr;
    std::vector<std::vector<GatherTask>> steps;
    auto at = [&](size_t t) -> std::vector<GatherTask> & {
        if (steps.size() <= t) steps.resize(t + 1);
        return steps[t];
    };
    for (auto &st : sw->strips) {
        const TableSet &ts = *st.tabs;
        const int r = st.r;
        const uint32_t *pr = sw->primes_dev + st.group * Pg;
        const int smax = st.heights.back();
        const int nf = (int)ts.row.size();  // launches per row (factors, or pairs of factors)
        // main lane: rows 1..smax-1, launch i of row h is step (h-1)*nf + i
        for (int row = 0; row < smax - 1; ++row)
            for (int i = 0; i < nf; ++i) {
                const size_t t = (size_t)row * nf + i;
                append_gather_tasks(&at(t), ts.row[i], st.vec[t & 1], st.vec[(t & 1) ^ 1], pr, sw->D1, Pg, true);
                count_work(sw, ts.row[i], Pg);
            }
        // read-out lanes
        for (int h : st.heights) {
            const size_t t0 = (size_t)(h - 1) * nf;
            const uint32_t *src = st.vec[t0 & 1];
            uint32_t *slot = sw->ptilde_dev + ((size_t)st.group * n_rects + rect_index(sw, r, h)) * row_words;
            int sc = 0;
            for (size_t i = 0; i < ts.last.size(); ++i) {
                const bool final = i + 1 == ts.last.size();
                uint32_t *dst = final ? slot : st.scratch[sc];
                append_gather_tasks(&at(t0 + i), ts.last[i], src, dst, pr, sw->D1, Pg, !final);
                count_work(sw, ts.last[i], Pg);
                src = dst;
                sc ^= 1;
            }
        }
    }
    std::vector<GatherTask> all;
    for (auto &l : steps) {
        const int et = effective_tile(l, tile);
        sw->step_off.push_back((uint32_t)all.size());
        sw->step_ntasks.push_back((uint32_t)l.size());
        sw->step_tile.push_back(et);
        sw->step_blocks.push_back(assign_blocks(l, et));
        all.insert(all.end(), l.begin(), l.end());
    }
    if ((rc = dev_alloc((void **)&sw->tasks_dev, std::max<size_t>(1, all.size()) * sizeof(GatherTask)))) return rc;
    CP_CUDA_TRY(cudaMemcpy(sw->tasks_dev, all.data(), all.size() * sizeof(GatherTask), cudaMemcpyHostToDevice));
    // capture the program into one graph
    CP_CUDA_TRY(cudaStreamBeginCapture(sw->stream, cudaStreamCaptureModeThreadLocal));
    rc = enqueue_program(sw);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(sw->stream, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(CP_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    sw->graph = g;
    CP_CUDA_TRY(cudaGraphInstantiate(&sw->exec, g, 0));
    return CP_OK;
}

// Enqueue the whole sweep on sw->stream (used once, under graph capture).
static int enqueue_program(cp_sweep *sw) {
    const size_t row_words = (size_t)sw->D1 * sw->Pg;
    for (auto &st : sw->strips) {  // vector := e_0 over the NCNNN input space of T_1
        CP_CUDA_TRY(cudaMemsetAsync(st.vec[0], 0, st.tabs->S_b * row_words * 4, sw->stream));
        CP_CUDA_TRY(cudaMemcpyAsync(st.vec[0], sw->ones_dev, 4 * sw->Pg, cudaMemcpyDeviceToDevice, sw->stream));
    }
    for (size_t t = 0; t < sw->step_off.size(); ++t) {
        int rc = launch_gather(sw->tasks_dev + sw->step_off[t], (int)sw->step_ntasks[t], sw->step_blocks[t],
                               sw->step_tile[t], sw->stream);
        if (rc) return rc;
    }
    SeriesParams sp{};
    sp.lattice = sw->lattice;
    sp.k = sw->k;
    sp.n = sw->n;
    sp.D1 = sw->D1;
    sp.P = sw->P;
    sp.Pg = sw->Pg;
    sp.n_rects = (int)sw->rects.size();
    sp.mmax = sw->k / 2;
    sp.add_mu = (sw->lattice == CP_SQUARE && sw->k % 2 == 1) ? 1 : 0;
    return launch_flm_series(sw->ptilde_dev, sw->rects_dev, sw->primes_dev, sp, sw->series_dev, sw->err_dev,
                             sw->stream);
}

static int sweep_build(int lattice, int k, const uint32_t *primes, int P, int tile, int groups, cudaStream_t stream,
                       cp_sweep **out) {
    auto sw = std::make_unique<cp_sweep>();
    sw->lattice = lattice;
    sw->k = k;
    sw->P = P;
    sw->n = n_terms_for(lattice, k);
    sw->D1 = sw->n;
    sw->groups = groups;
    sw->Pg = P / groups;
    sw->stream = stream;
    int rc;
    if ((rc = prepare_gather_kernels()) || (rc = crt_static_touch())) return rc;
    sw->primes_host.assign(primes, primes + P);
    if ((rc = dev_alloc((void **)&sw->primes_dev, 4 * CP_MAX_PRIMES))) return rc;
    CP_CUDA_TRY(cudaMemcpy(sw->primes_dev, primes, 4 * P, cudaMemcpyHostToDevice));
    std::vector<uint32_t> ones(CP_MAX_PRIMES, 1u);
    if ((rc = dev_alloc((void **)&sw->ones_dev, 4 * CP_MAX_PRIMES))) return rc;
    CP_CUDA_TRY(cudaMemcpy(sw->ones_dev, ones.data(), 4 * CP_MAX_PRIMES, cudaMemcpyHostToDevice));
    int n_rects = 0;
    for (int r = 1; 2 * r <= k; ++r)
        for (int s = r; r + s <= k; ++s)
            if (r + s >= k - 3) ++n_rects;
    if ((rc = dev_alloc((void **)&sw->ptilde_dev, 4ull * n_rects * sw->D1 * P))) return rc;
    if ((rc = dev_alloc((void **)&sw->series_dev, 4ull * 3 * P * sw->n))) return rc;
    if ((rc = dev_alloc((void **)&sw->err_dev, sizeof(int)))) return rc;
    CP_CUDA_TRY(cudaMemset(sw->err_dev, 0, sizeof(int)));
    if ((rc = build_strips(sw.get()))) return rc;
    if ((rc = dev_alloc((void **)&sw->rects_dev, sizeof(int2) * n_rects))) return rc;
    CP_CUDA_TRY(cudaMemcpy(sw->rects_dev, sw->rects.data(), sizeof(int2) * n_rects, cudaMemcpyHostToDevice));
    if ((rc = build_program(sw.get(), tile))) return rc;
    *out = sw.release();
    return CP_OK;
}

static int sweep_time_once(cp_sweep *sw, float *ms) {
    cudaEvent_t a, b;
    CP_CUDA_TRY(cudaEventCreate(&a));
    CP_CUDA_TRY(cudaEventCreate(&b));
    cudaError_t e = cudaGraphLaunch(sw->exec, sw->stream);  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(a, sw->stream);
    if (e == cudaSuccess) e = cudaGraphLaunch(sw->exec, sw->stream);
    if (e == cudaSuccess) e = cudaEventRecord(b, sw->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return fail(CP_ECUDA, std::string("autotune timing: ") + cudaGetErrorString(e));
    return CP_OK;
}

static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int, int>, std::pair<int, int>> g_tuned;  // (dev, lattice, k, P) -> (tile, groups)

extern "C" int cp_sweep_create(int lattice, int k, const uint32_t *primes, int n_primes, int tile, int prime_groups,
                               void *cuda_stream, cp_sweep **out) {
    if (!out) return fail(CP_EINVAL, "out is NULL");
    *out = nullptr;
    if (lattice != CP_SQUARE && lattice != CP_TRIANGULAR) return fail(CP_EINVAL, "bad lattice");
    if (k < 4 || k / 2 > CP_MAX_L) return fail(CP_EINVAL, "k must satisfy 4 <= k and k/2 <= CP_MAX_L");
    if (n_terms_for(lattice, k) > kMaxSeries) return fail(CP_EINVAL, "k too large for the series kernel");
    int rc = check_primes(primes, n_primes);
    if (rc) return rc;
    if (!cuda_stream) return fail(CP_EINVAL, "the sweep needs a non-default stream (graph capture)");
    {
        const int rows = tile & 0xFFF, ring = (tile >> 12) & 0xFF, edges = (tile >> 20) & 15,
                  cpt = (tile >> 24) & 15;
        const bool reg = (rows == 1 || rows == 2 || rows == 4 || rows == 8) && (tile >> 12) == 0;
        const bool tma = (rows == 16 || rows == 32 || rows == 64 || rows == 128) && (tile >> 30) == 0 && tile_shape(tile) != 3 &&
                         (cpt <= 2 || cpt == 4) &&
                         (ring == 0 || (ring >= 16 && ring <= 192)) &&
                         (edges <= 2 || edges == 4 || edges == 8);
        if (tile != 0 && !reg && !tma)
            return fail(CP_EINVAL, "tile must be 0 (autotune), 1, 2, 4, 8 (register kernel) or 16, 32, 64, 128 "
                                   "(TMA) + (ring KB 16..192 << 12) + (edges per stage 1, 2, 4, 8 << 20) + "
                                   "(chunks per thread 1, 2, 4 << 24) + (block shape 1 wide, 2 narrow << 28)");
    }
    if (prime_groups < 0 || (prime_groups > 0 && n_primes % prime_groups != 0))
        return fail(CP_EINVAL, "prime_groups must divide n_primes");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (tile != 0 && prime_groups != 0) return sweep_build(lattice, k, primes, n_primes, tile, prime_groups, st, out);
    int dev = 0;
    CP_CUDA_TRY(cudaGetDevice(&dev));
    auto key = std::make_tuple(dev, lattice, k, n_primes);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end())
            return sweep_build(lattice, k, primes, n_primes, tile ? tile : it->second.first,
                               prime_groups ? prime_groups : it->second.second, st, out);
    }
    // autotune: for each prime grouping build the strips once, re-tile the
    // launch program for each candidate tile, time one graph run (after a
    // warm-up run) and keep the fastest (tile, grouping)
    std::vector<int> tiles = tile ? std::vector<int>{tile}
                                  : std::vector<int>{make_tile(32, 0, 0, 0), make_tile(64, 0, 0, 0),
                                                     make_tile(32, 48, 4, 2), make_tile(64, 48, 4, 2),
                                                     make_tile(32, 64, 8, 1) | kTileWide,
                                                     make_tile(64, 64, 8, 1) | kTileWide,
                                                     make_tile(16, 0, 0, 0), 4};
    std::vector<int> grps;
    if (prime_groups) grps = {prime_groups};
    else
        for (int g : {1, 2})
            if (n_primes % g == 0 && (n_primes / g) % 4 == 0) grps.push_back(g);
    if (grps.empty()) grps = {1};
    float best = 1e30f;
    int bt = tiles[0], bg = grps[0];
    for (int g : grps) {
        cp_sweep *cand = nullptr;
        if ((rc = sweep_build(lattice, k, primes, n_primes, tiles[0], g, st, &cand))) return rc;
        for (size_t ti = 0; ti < tiles.size(); ++ti) {
            if (ti > 0 && (rc = build_program(cand, tiles[ti]))) break;
            float ms = 0;
            if ((rc = sweep_time_once(cand, &ms))) break;
            if ((rc = check_device_error(st))) break;
            if (ms < best) {
                best = ms;
                bt = tiles[ti];
                bg = g;
            }
        }
        delete cand;
        if (rc) return rc;
    }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[key] = {bt, bg};
    }
    return sweep_build(lattice, k, primes, n_primes, bt, bg, st, out);
}

extern "C" int cp_sweep_run(cp_sweep *sw) {
    if (!sw) return fail(CP_EINVAL, "sweep is NULL");
    CP_CUDA_TRY(cudaGraphLaunch(sw->exec, sw->stream));
    return CP_OK;
}

extern "C" int cp_sweep_sync(cp_sweep *sw) {
    if (!sw) return fail(CP_EINVAL, "sweep is NULL");
    CP_CUDA_TRY(cudaStreamSynchronize(sw->stream));
    int rc = check_device_error(sw->stream);
    if (rc) return rc;
    int herr = 0;
    CP_CUDA_TRY(cudaMemcpy(&herr, sw->err_dev, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr) return fail(CP_ESTATE, "a rectangle's P~ lacks constant term 1");
    return CP_OK;
}

extern "C" int cp_sweep_work(const cp_sweep *sw, uint64_t work[3]) {
    if (!sw || !work) return fail(CP_EINVAL, "NULL argument");
    work[0] = sw->updates;
    work[1] = sw->bytes;
    work[2] = sw->site_bytes;
    return CP_OK;
}

extern "C" int cp_sweep_info(const cp_sweep *sw, int *n_rects, int *n_terms, int *tile, int *prime_groups,
                             uint64_t *updates_per_run, uint64_t *bytes_per_run, int *launches_per_run) {
    if (!sw) return fail(CP_EINVAL, "sweep is NULL");
    if (n_rects) *n_rects = (int)sw->rects.size();
    if (n_terms) *n_terms = sw->n;
    if (tile) *tile = sw->tile;
    if (prime_groups) *prime_groups = sw->groups;
    if (updates_per_run) *updates_per_run = sw->updates;
    if (bytes_per_run) *bytes_per_run = sw->bytes;
    if (launches_per_run) *launches_per_run = (int)sw->step_off.size() + 1;
    return CP_OK;
}

extern "C" int cp_sweep_rects(const cp_sweep *sw, int *rs_host, int max_rects) {
    if (!sw || !rs_host) return fail(CP_EINVAL, "NULL argument");
    if (max_rects < (int)sw->rects.size()) return fail(CP_EINVAL, "max_rects too small");
    for (size_t j = 0; j < sw->rects.size(); ++j) {
        rs_host[2 * j] = sw->rects[j].x;
        rs_host[2 * j + 1] = sw->rects[j].y;
    }
    return CP_OK;
}

extern "C" int cp_sweep_read_ptilde(cp_sweep *sw, uint32_t *out_host, size_t out_len) {
    if (!sw || !out_host) return fail(CP_EINVAL, "NULL argument");
    const int nr = (int)sw->rects.size(), D1 = sw->D1, Pg = sw->Pg;
    if (out_len < (size_t)nr * sw->P * D1) return fail(CP_EINVAL, "out_len < n_rects*n_primes*n_terms");
    std::vector<uint32_t> raw((size_t)sw->groups * nr * D1 * Pg);
    CP_CUDA_TRY(cudaStreamSynchronize(sw->stream));
    CP_CUDA_TRY(cudaMemcpy(raw.data(), sw->ptilde_dev, raw.size() * 4, cudaMemcpyDeviceToHost));
    for (int g = 0; g < sw->groups; ++g)
        for (int j = 0; j < nr; ++j)
            for (int d = 0; d < D1; ++d)
                for (int q = 0; q < Pg; ++q)
                    out_host[((size_t)j * sw->P + g * Pg + q) * D1 + d] = raw[(((size_t)g * nr + j) * D1 + d) * Pg + q];
    return CP_OK;
}

extern "C" int cp_sweep_read_series(cp_sweep *sw, uint32_t *out_host, size_t out_len) {
    if (!sw || !out_host) return fail(CP_EINVAL, "NULL argument");
    if (out_len < 3ull * sw->P * sw->n) return fail(CP_EINVAL, "out_len < 3*n_primes*n_terms");
    int rc = cp_sweep_sync(sw);
    if (rc) return rc;
    CP_CUDA_TRY(cudaMemcpy(out_host, sw->series_dev, 12ull * sw->P * sw->n, cudaMemcpyDeviceToHost));
    return CP_OK;
}

extern "C" int cp_sweep_read_series_device(cp_sweep *sw, uint32_t *out_dev, size_t out_len) {
    if (!sw || !out_dev) return fail(CP_EINVAL, "NULL argument");
    if (out_len < 3ull * sw->P * sw->n) return fail(CP_EINVAL, "out_len < 3*n_primes*n_terms");
    CP_CUDA_TRY(cudaMemcpyAsync(out_dev, sw->series_dev, 12ull * sw->P * sw->n, cudaMemcpyDeviceToDevice, sw->stream));
    return CP_OK;
}

extern "C" int cp_sweep_set_primes(cp_sweep *sw, const uint32_t *primes, int n_primes) {
    if (!sw) return fail(CP_EINVAL, "sweep is NULL");
    if (n_primes != sw->P) return fail(CP_EINVAL, "n_primes differs from the sweep's");
    int rc = check_primes(primes, n_primes);
    if (rc) return rc;
    CP_CUDA_TRY(cudaMemcpyAsync(sw->primes_dev, primes, 4ull * n_primes, cudaMemcpyHostToDevice, sw->stream));
    sw->primes_host.assign(primes, primes + n_primes);
    return CP_OK;
}

extern "C" int cp_sweep_series_integers(cp_sweep *sw, uint32_t *limbs_out, size_t limbs_len, int limbs_per_coeff,
                                        uint32_t *flags_out) {
    if (!sw || !limbs_out) return fail(CP_EINVAL, "NULL argument");
    const int n = sw->n, P = sw->P;
    if (limbs_per_coeff < 1 || limbs_len < 3ull * n * limbs_per_coeff)
        return fail(CP_EINVAL, "limbs_len < 3*n_terms*limbs_per_coeff");
    int rc;
    const size_t need = 3ull * n * (limbs_per_coeff + 1);
    if (need > sw->crt_words) {
        CP_CUDA_TRY(cudaStreamSynchronize(sw->stream));
        dev_free(sw->crt_dev);
        sw->crt_dev = nullptr;
        sw->crt_words = 0;
        if ((rc = dev_alloc((void **)&sw->crt_dev, need * 4))) return rc;
        sw->crt_words = need;
    }
    uint32_t *limbs_d = sw->crt_dev, *flags_d = limbs_d + 3ull * n * limbs_per_coeff;
    for (int x = 0; x < 3; ++x)
        if ((rc = launch_crt(sw->series_dev + (size_t)x * P * n, sw->primes_host.data(), P, n,
                             limbs_d + (size_t)x * n * limbs_per_coeff, limbs_per_coeff, nullptr, flags_d + (size_t)x * n,
                             sw->stream)))
            return rc;
    std::vector<uint32_t> flags(3ull * n);
    CP_CUDA_TRY(cudaMemcpyAsync(limbs_out, limbs_d, 12ull * n * limbs_per_coeff, cudaMemcpyDeviceToHost, sw->stream));
    CP_CUDA_TRY(cudaMemcpyAsync(flags.data(), flags_d, 12ull * n, cudaMemcpyDeviceToHost, sw->stream));
    if ((rc = cp_sweep_sync(sw))) return rc;
    if (flags_out)
        for (size_t j = 0; j < flags.size(); ++j) flags_out[j] = flags[j];
    return crt_outcome(flags.data(), 3 * n);
}

// The same program without the graph, with an event pair around every batched
// gather launch: sum of gather kernel times and number of gather launches.
extern "C" int cp_sweep_profile(cp_sweep *sw, float *gather_ms, int *n_gather, float *total_ms) {
    if (!sw) return fail(CP_EINVAL, "sweep is NULL");
    const size_t nst = sw->step_off.size();
    std::vector<cudaEvent_t> ev(2 * nst + 2);
    for (auto &e : ev) CP_CUDA_TRY(cudaEventCreate(&e));
    const size_t row_words = (size_t)sw->D1 * sw->Pg;
    int rc = CP_OK;
    CP_CUDA_TRY(cudaEventRecord(ev[2 * nst], sw->stream));
    for (auto &st : sw->strips) {
        CP_CUDA_TRY(cudaMemsetAsync(st.vec[0], 0, st.tabs->S_b * row_words * 4, sw->stream));
        CP_CUDA_TRY(cudaMemcpyAsync(st.vec[0], sw->ones_dev, 4 * sw->Pg, cudaMemcpyDeviceToDevice, sw->stream));
    }
    for (size_t t = 0; t < nst && rc == CP_OK; ++t) {
        cudaEventRecord(ev[2 * t], sw->stream);
        rc = launch_gather(sw->tasks_dev + sw->step_off[t], (int)sw->step_ntasks[t], sw->step_blocks[t],
                           sw->step_tile[t], sw->stream);
        cudaEventRecord(ev[2 * t + 1], sw->stream);
    }
    CP_CUDA_TRY(cudaEventRecord(ev[2 * nst + 1], sw->stream));
    cudaError_t e = cudaEventSynchronize(ev[2 * nst + 1]);
    float sum = 0, tot = 0;
    for (size_t t = 0; t < nst && e == cudaSuccess; ++t) {
        float ms = 0;
        e = cudaEventElapsedTime(&ms, ev[2 * t], ev[2 * t + 1]);
        sum += ms;
    }
    if (e == cudaSuccess) e = cudaEventElapsedTime(&tot, ev[2 * nst], ev[2 * nst + 1]);
    for (auto &x : ev) cudaEventDestroy(x);
    if (rc) return rc;
    if (e != cudaSuccess) return fail(CP_ECUDA, std::string("profile: ") + cudaGetErrorString(e));
    if (gather_ms) *gather_ms = sum;
    if (n_gather) *n_gather = (int)nst;
    if (total_ms) *total_ms = tot;
    return CP_OK;
}

extern "C" void cp_sweep_destroy(cp_sweep *sw) {
    if (!sw) return;
    cudaStreamSynchronize(sw->stream);
    delete sw;
}
