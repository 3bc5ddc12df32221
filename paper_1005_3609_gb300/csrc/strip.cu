// cp_strip: one L-wide strip advanced row by row (eq. (Z_from_T)), with the
// C-ABI entry points declared in cp_tm.h.
#include <cuda_runtime.h>

#include <cstring>
#include <string>
#include <vector>

#include "cp_internal.h"

namespace cp {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }

int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

int dev_alloc(void **p, size_t bytes) {
    *p = nullptr;
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? CP_ENOMEM : CP_ECUDA,
                    "cudaMalloc(" + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    }
    return CP_OK;
}

void dev_free(void *p) {
    if (p) cudaFree(p);
}

// Deterministic Miller-Rabin for n < 2^32 (bases 2, 7, 61).
static bool host_is_prime(uint32_t n) {
    if (n < 2) return false;
    for (uint32_t q : {2u, 3u, 5u, 7u, 11u, 13u, 17u, 19u, 23u, 29u, 31u, 37u, 61u}) {
        if (n == q) return true;
        if (n % q == 0) return false;
    }
    uint32_t d = n - 1;
    int r = 0;
    while (!(d & 1)) { d >>= 1; ++r; }
    auto mul = [n](uint64_t a, uint64_t b) { return (a * b) % n; };
    for (uint64_t a : {2ull, 7ull, 61ull}) {
        uint64_t x = 1, b = a % n;
        for (uint32_t e = d; e; e >>= 1, b = mul(b, b))
            if (e & 1) x = mul(x, b);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int k = 1; k < r && comp; ++k) {
            x = mul(x, x);
            if (x == n - 1) comp = false;
        }
        if (comp) return false;
    }
    return true;
}

int check_primes(const uint32_t *primes, int n) {
    if (!primes || n < 1 || n > CP_MAX_PRIMES) return fail(CP_EINVAL, "n_primes must be 1..CP_MAX_PRIMES");
    for (int k = 0; k < n; ++k) {
        uint32_t p = primes[k];
        if (p < 2 || p >= (1u << 31)) return fail(CP_EINVAL, "prime out of range [2, 2^31)");
        if (!host_is_prime(p)) return fail(CP_EINVAL, "not a prime: " + std::to_string(p));
        for (int j = 0; j < k; ++j)
            if (primes[j] == p) return fail(CP_EINVAL, "duplicate prime");
    }
    return CP_OK;
}

}  // namespace cp

using namespace cp;

struct cp_strip {
    int lattice = 0, L = 0, P = 0, D1 = 0, max_rows = 0, height = 1;
    cudaStream_t stream = nullptr;
    std::shared_ptr<TableSet> tabs;
    uint32_t *primes_dev = nullptr;
    uint32_t *vec[2] = {nullptr, nullptr};
    int cur = 0;
    uint32_t *scratch[2] = {nullptr, nullptr};
    uint32_t *row_out = nullptr;  // [P][D1]
    uint32_t *ones_dev = nullptr;  // P ones (the e_0 row)
    uint32_t *crt_dev = nullptr;   // cp_read_integers: limbs, then flags, then bounds (grown on demand)
    size_t crt_words = 0;
    GatherTask *tasks_dev = nullptr;
    int tile = kGatherItems;  // gather tile of this strip's launches
    // precomputed launches: row factors from vec[0] / vec[1], read-out chain
    std::vector<std::vector<GatherTask>> row_tasks[2];
    std::vector<std::vector<GatherTask>> last_tasks[2];
    std::vector<GatherTask *> row_dev[2], last_dev[2];
    const uint32_t *last_result[2] = {nullptr, nullptr};

    ~cp_strip() {
        dev_free(primes_dev);
        dev_free(vec[0]);
        dev_free(vec[1]);
        dev_free(scratch[0]);
        dev_free(scratch[1]);
        dev_free(row_out);
        dev_free(ones_dev);
        dev_free(tasks_dev);
        dev_free(crt_dev);
    }
};

static int upload_tasks(cp_strip *s, std::vector<std::vector<GatherTask>> &lists, std::vector<GatherTask *> &ptrs,
                        std::vector<GatherTask> &all) {
    for (auto &l : lists) {
        assign_blocks(l, s->tile);
        ptrs.push_back(reinterpret_cast<GatherTask *>(all.size()));  // offset, fixed up later
        all.insert(all.end(), l.begin(), l.end());
    }
    return CP_OK;
}

static uint32_t list_blocks(const std::vector<GatherTask> &l, int tile) {
    uint32_t n = 0;
    for (auto &t : l) n += task_blocks(t, tile);
    return n;
}

static int check_strip_args(int lattice, int L, const uint32_t *primes, int n_primes, int max_degree, int max_rows,
                            cp_strip **out) {
    if (!out) return fail(CP_EINVAL, "out is NULL");
    *out = nullptr;
    if (lattice != CP_SQUARE && lattice != CP_TRIANGULAR) return fail(CP_EINVAL, "lattice must be CP_SQUARE or CP_TRIANGULAR");
    if (L < 1 || L > CP_MAX_L) return fail(CP_EINVAL, "L must be 1..CP_MAX_L");
    if (max_rows < 1) return fail(CP_EINVAL, "max_rows must be >= 1");
    if (max_degree < -1) return fail(CP_EINVAL, "max_degree must be >= -1");
    int rc = check_primes(primes, n_primes);
    if (rc) return rc;
    long long D = max_degree >= 0 ? max_degree : (long long)L * max_rows - 1;
    if (D + 1 > (1 << 20)) return fail(CP_EINVAL, "degree too large");
    return CP_OK;
}

// The strip around a table set: state vectors, read-out scratch, precomputed launches.
static int make_strip(std::shared_ptr<TableSet> tabs, int lattice, int L, const uint32_t *primes, int n_primes,
                      int max_degree, int max_rows, void *cuda_stream, cp_strip **out) {
    int rc = CP_OK;
    long long D = max_degree >= 0 ? max_degree : (long long)L * max_rows - 1;
    auto s = std::make_unique<cp_strip>();
    s->lattice = lattice;
    s->L = L;
    s->P = n_primes;
    s->D1 = (int)D + 1;
    s->max_rows = max_rows;
    s->stream = (cudaStream_t)cuda_stream;
    s->tabs = std::move(tabs);
    const TableSet &ts = *s->tabs;
    const size_t row_words = (size_t)s->D1 * s->P;
    if ((rc = dev_alloc((void **)&s->primes_dev, 4 * CP_MAX_PRIMES))) return rc;
    CP_CUDA_TRY(cudaMemcpy(s->primes_dev, primes, 4 * n_primes, cudaMemcpyHostToDevice));
    for (int k = 0; k < 2; ++k)
        if ((rc = dev_alloc((void **)&s->vec[k], ts.S_max * row_words * 4))) return rc;
    // read-out scratch: T_1^last writes cnt[L-1] rows, T_2^last cnt[L-2], ...
    uint64_t sA = ts.last[0].n_dst, sB = ts.last.size() >= 2 ? ts.last[1].n_dst : 1;
    if ((rc = dev_alloc((void **)&s->scratch[0], sA * row_words * 4))) return rc;
    if ((rc = dev_alloc((void **)&s->scratch[1], sB * row_words * 4))) return rc;
    if ((rc = dev_alloc((void **)&s->row_out, row_words * 4))) return rc;
    // TMA gather when the rows are 16-byte chunked and fit the ring, else the register kernel
    {
        std::vector<GatherTask> probe;
        append_gather_tasks(&probe, ts.row[0], s->vec[0], s->vec[1], s->primes_dev, s->D1, s->P);
        s->tile = effective_tile(probe, make_tile(default_rows(probe), 0, 0, 0));
    }
    // launches of one row (starting from vec[b]) and of the read-out chain from vec[b]
    std::vector<GatherTask> all;
    for (int b = 0; b < 2; ++b) {
        int cur = b;
        for (size_t i = 0; i < ts.row.size(); ++i) {
            std::vector<GatherTask> l;
            append_gather_tasks(&l, ts.row[i], s->vec[cur], s->vec[cur ^ 1], s->primes_dev, s->D1, s->P, true);
            s->row_tasks[b].push_back(l);
            cur ^= 1;
        }
        const uint32_t *src = s->vec[b];
        int sc = 0;
        for (size_t i = 0; i < ts.last.size(); ++i) {
            std::vector<GatherTask> l;
            append_gather_tasks(&l, ts.last[i], src, s->scratch[sc], s->primes_dev, s->D1, s->P,
                                i + 1 < ts.last.size());
            s->last_tasks[b].push_back(l);
            src = s->scratch[sc];
            sc ^= 1;
        }
        s->last_result[b] = src;
        upload_tasks(s.get(), s->row_tasks[b], s->row_dev[b], all);
        upload_tasks(s.get(), s->last_tasks[b], s->last_dev[b], all);
    }
    if ((rc = dev_alloc((void **)&s->tasks_dev, all.size() * sizeof(GatherTask)))) return rc;
    CP_CUDA_TRY(cudaMemcpy(s->tasks_dev, all.data(), all.size() * sizeof(GatherTask), cudaMemcpyHostToDevice));
    for (int b = 0; b < 2; ++b) {
        for (auto &p : s->row_dev[b]) p = s->tasks_dev + reinterpret_cast<size_t>(p);
        for (auto &p : s->last_dev[b]) p = s->tasks_dev + reinterpret_cast<size_t>(p);
    }
    // e_0: rank 0 of the NCNNN space, polynomial 1
    std::vector<uint32_t> one(s->P, 1u);
    if ((rc = dev_alloc((void **)&s->ones_dev, 4 * s->P))) return rc;
    CP_CUDA_TRY(cudaMemcpy(s->ones_dev, one.data(), 4 * s->P, cudaMemcpyHostToDevice));
    CP_CUDA_TRY(cudaMemsetAsync(s->vec[0], 0, ts.S_max * row_words * 4, s->stream));
    CP_CUDA_TRY(cudaMemcpyAsync(s->vec[0], s->ones_dev, 4 * s->P, cudaMemcpyDeviceToDevice, s->stream));
    CP_CUDA_TRY(cudaStreamSynchronize(s->stream));
    s->cur = 0;
    s->height = 1;
    *out = s.release();
    return CP_OK;
}

extern "C" int cp_create_strip(int lattice, int L, const uint32_t *primes, int n_primes, int max_degree,
                               int max_rows, void *cuda_stream, cp_strip **out) {
    int rc = check_strip_args(lattice, L, primes, n_primes, max_degree, max_rows, out);
    if (rc) return rc;
    if ((rc = prepare_gather_kernels()) || (rc = crt_static_touch())) return rc;
    std::shared_ptr<TableSet> tabs;
    const long long D1 = max_degree >= 0 ? max_degree + 1 : (long long)L * max_rows;
    if ((rc = get_tables(lattice, L, (size_t)D1 * n_primes * 4, (cudaStream_t)cuda_stream, &tabs))) return rc;
    return make_strip(std::move(tabs), lattice, L, primes, n_primes, max_degree, max_rows, cuda_stream, out);
}

extern "C" int cp_create_strip_potts(int lattice, int L, int v, const uint32_t *primes, int n_primes, int max_degree,
                                     int max_rows, void *cuda_stream, cp_strip **out) {
    int rc = check_strip_args(lattice, L, primes, n_primes, max_degree, max_rows, out);
    if (rc) return rc;
    if (v < -CP_POTTS_MAX_V || v > CP_POTTS_MAX_V) return fail(CP_EINVAL, "v must be in [-CP_POTTS_MAX_V, CP_POTTS_MAX_V]");
    if (L > CP_POTTS_MAX_L) return fail(CP_EINVAL, "L must be 1..CP_POTTS_MAX_L for the Potts strip");
    if ((rc = prepare_gather_kernels()) || (rc = crt_static_touch())) return rc;
    std::shared_ptr<TableSet> tabs;
    if ((rc = get_potts_tables(lattice, L, v, (cudaStream_t)cuda_stream, &tabs))) return rc;
    return make_strip(std::move(tabs), lattice, L, primes, n_primes, max_degree, max_rows, cuda_stream, out);
}

extern "C" int cp_advance_rows(cp_strip *s, int n_rows) {
    if (!s) return fail(CP_EINVAL, "strip is NULL");
    if (n_rows < 0 || (long long)s->height + n_rows > s->max_rows) return fail(CP_EINVAL, "height would exceed max_rows");
    for (int r = 0; r < n_rows; ++r) {
        const int b = s->cur;
        const int nrow = (int)s->row_tasks[b].size();
        for (int i = 0; i < nrow; ++i) {
            int rc = launch_gather(s->row_dev[b][i], (int)s->row_tasks[b][i].size(),
                                   list_blocks(s->row_tasks[b][i], s->tile), s->tile, s->stream);
            if (rc) return rc;
        }
        s->cur = (b + nrow) & 1;
        s->height += 1;
    }
    return CP_OK;
}

static int readout(cp_strip *s) {
    const int b = s->cur;
    for (size_t i = 0; i < s->last_tasks[b].size(); ++i) {
        int rc = launch_gather(s->last_dev[b][i], (int)s->last_tasks[b][i].size(),
                               list_blocks(s->last_tasks[b][i], s->tile), s->tile, s->stream);
        if (rc) return rc;
    }
    return launch_transpose_row(s->last_result[b], s->row_out, s->D1, s->P, s->stream);
}

extern "C" int cp_read_coeffs_device(cp_strip *s, uint32_t *out_dev, size_t out_len) {
    if (!s || !out_dev) return fail(CP_EINVAL, "NULL argument");
    if (out_len < (size_t)s->P * s->D1) return fail(CP_EINVAL, "out_len < n_primes*(D+1)");
    int rc = readout(s);
    if (rc) return rc;
    CP_CUDA_TRY(cudaMemcpyAsync(out_dev, s->row_out, 4ull * s->P * s->D1, cudaMemcpyDeviceToDevice, s->stream));
    return CP_OK;
}

extern "C" int cp_read_coeffs(cp_strip *s, uint32_t *out, size_t out_len, int *height_out) {
    if (!s || !out) return fail(CP_EINVAL, "NULL argument");
    if (out_len < (size_t)s->P * s->D1) return fail(CP_EINVAL, "out_len < n_primes*(D+1)");
    int rc = readout(s);
    if (rc) return rc;
    CP_CUDA_TRY(cudaMemcpyAsync(out, s->row_out, 4ull * s->P * s->D1, cudaMemcpyDeviceToHost, s->stream));
    if ((rc = check_device_error(s->stream))) return rc;
    if (height_out) *height_out = s->height;
    return CP_OK;
}

extern "C" int cp_read_integers(cp_strip *s, uint32_t *limbs_out, size_t limbs_len, int limbs_per_coeff,
                                uint32_t *flags_out, int *height_out) {
    if (!s || !limbs_out) return fail(CP_EINVAL, "NULL argument");
    const int D1 = s->D1;
    if (limbs_per_coeff < 1 || limbs_len < (size_t)D1 * limbs_per_coeff)
        return fail(CP_EINVAL, "limbs_len < (D+1)*limbs_per_coeff");
    // Whitney's bound |c_j| <= C(|E|, j) of the chromatic polynomial; the Potts
    // strip's coefficients have no such bound, only the stabilisation check
    const bool bound = !s->tabs->potts;
    std::vector<uint32_t> bits(D1, 0u);
    if (bound) binomial_bits(rectangle_edges(s->lattice, s->L, s->height), D1, bits.data());
    const size_t need = (size_t)D1 * (limbs_per_coeff + 2);
    int rc;
    if (need > s->crt_words) {
        CP_CUDA_TRY(cudaStreamSynchronize(s->stream));
        dev_free(s->crt_dev);
        s->crt_dev = nullptr;
        s->crt_words = 0;
        if ((rc = dev_alloc((void **)&s->crt_dev, need * 4))) return rc;
        s->crt_words = need;
    }
    uint32_t *limbs_d = s->crt_dev, *flags_d = limbs_d + (size_t)D1 * limbs_per_coeff, *bound_d = flags_d + D1;
    if ((rc = readout(s))) return rc;
    CP_CUDA_TRY(cudaMemcpyAsync(bound_d, bits.data(), 4ull * D1, cudaMemcpyHostToDevice, s->stream));
    std::vector<uint32_t> primes(s->P);
    CP_CUDA_TRY(cudaMemcpyAsync(primes.data(), s->primes_dev, 4ull * s->P, cudaMemcpyDeviceToHost, s->stream));
    CP_CUDA_TRY(cudaStreamSynchronize(s->stream));
    if ((rc = launch_crt(s->row_out, primes.data(), s->P, D1, limbs_d, limbs_per_coeff, bound ? bound_d : nullptr,
                         flags_d, s->stream)))
        return rc;
    std::vector<uint32_t> flags(D1);
    CP_CUDA_TRY(cudaMemcpyAsync(limbs_out, limbs_d, 4ull * D1 * limbs_per_coeff, cudaMemcpyDeviceToHost, s->stream));
    CP_CUDA_TRY(cudaMemcpyAsync(flags.data(), flags_d, 4ull * D1, cudaMemcpyDeviceToHost, s->stream));
    if ((rc = check_device_error(s->stream))) return rc;
    if (flags_out)
        for (int j = 0; j < D1; ++j) flags_out[j] = flags[j];
    if (height_out) *height_out = s->height;
    return crt_outcome(flags.data(), D1);
}

extern "C" int cp_strip_info(const cp_strip *s, uint64_t n_states[2], int *degree, int *height) {
    if (!s) return fail(CP_EINVAL, "strip is NULL");
    if (n_states) {
        n_states[0] = s->tabs->S_b;
        n_states[1] = s->tabs->S_max;
    }
    if (degree) *degree = s->D1 - 1;
    if (height) *height = s->height;
    return CP_OK;
}

extern "C" int cp_strip_work(const cp_strip *s, uint64_t work[6]) {
    if (!s || !work) return fail(CP_EINVAL, "NULL argument");
    const uint64_t row = (uint64_t)s->D1 * s->P;  // words per state
    for (int k = 0; k < 6; ++k) work[k] = 0;
    // updates, own bytes, one-factor-at-a-time bytes -> work[u], work[b], work[f]
    auto add = [&](const SiteTable &t, int u, int b, int f) {
        const uint64_t mid = t.n_site_out - t.n_dst;  // intermediate states of a two-site table
        const uint64_t csr = 4 * (t.n_dst + 1 + t.nnz);
        work[u] += t.n_site_out * row;
        work[b] += 4 * (t.n_src + t.n_dst) * row + csr;
        work[f] += 4 * (t.n_src + 2 * mid + t.n_dst) * row + csr;
    };
    for (const SiteTable &t : s->tabs->row) add(t, 0, 1, 4);
    for (const SiteTable &t : s->tabs->last) add(t, 2, 3, 5);
    return CP_OK;
}

extern "C" int cp_strip_set_tile(cp_strip *s, int tile) {
    if (!s) return fail(CP_EINVAL, "strip is NULL");
    const int rows = tile & 0xFFF, ring = (tile >> 12) & 0xFF, edges = (tile >> 20) & 15, cpt = (tile >> 24) & 15;
    const bool reg = (rows == 1 || rows == 2 || rows == 4 || rows == 8) && (tile >> 12) == 0;
    const bool tma = (rows == 16 || rows == 32 || rows == 64 || rows == 128) && (tile >> 30) == 0 && tile_shape(tile) != 3 &&
                     (ring == 0 || (ring >= 16 && ring <= 192)) && (edges <= 2 || edges == 4 || edges == 8) &&
                     (cpt <= 2 || cpt == 4);
    if (tile != 0 && !reg && !tma) return fail(CP_EINVAL, "bad tile (encoding as for cp_sweep_create)");
    const int t = effective_tile(s->row_tasks[0][0],
                                 tile ? tile : make_tile(default_rows(s->row_tasks[0][0]), 0, 0, 0));
    CP_CUDA_TRY(cudaStreamSynchronize(s->stream));
    s->tile = t;
    std::vector<GatherTask> all;
    std::vector<GatherTask *> unused;
    for (int b = 0; b < 2; ++b) {
        upload_tasks(s, s->row_tasks[b], unused, all);
        upload_tasks(s, s->last_tasks[b], unused, all);
    }
    CP_CUDA_TRY(cudaMemcpy(s->tasks_dev, all.data(), all.size() * sizeof(GatherTask), cudaMemcpyHostToDevice));
    return CP_OK;
}

extern "C" int cp_strip_reset(cp_strip *s) {
    if (!s) return fail(CP_EINVAL, "strip is NULL");
    const size_t row_words = (size_t)s->D1 * s->P;
    CP_CUDA_TRY(cudaMemsetAsync(s->vec[0], 0, s->tabs->S_b * row_words * 4, s->stream));
    CP_CUDA_TRY(cudaMemcpyAsync(s->vec[0], s->ones_dev, 4 * s->P, cudaMemcpyDeviceToDevice, s->stream));
    s->cur = 0;
    s->height = 1;
    return CP_OK;
}

extern "C" void cp_destroy(cp_strip *s) {
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream); else cudaDeviceSynchronize();
    delete s;
}

extern "C" const char *cp_last_error(void) { return g_err.c_str(); }

namespace cp {
void clear_table_cache();
}
extern "C" void cp_clear_table_cache(void) { cp::clear_table_cache(); }

extern "C" int cp_set_factor_pairing(int on) { return cp::set_factor_pairing(on); }
