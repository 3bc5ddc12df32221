// The per-site operator kernel: one sparse factor T_i (or T_i^last) applied to
// a state vector, as a gather over the factor's CSR-by-destination table.
//
//   out[dst][d][p] = sum_{e in CSR(dst)} coef_e * in[src_e][d - shift_e][p]   (mod p)
//
// with in[..][d < 0] = 0 and degrees above D dropped: multiplying by w = 1/q
// is a shift of the coefficient index (Sec. 3.1, 3.5).  Rows are laid out
// [state][degree][prime], so a shift by one degree is a shift by n_primes
// words and, for n_primes % 4 == 0, every access is an aligned 16-byte load
// that reads four primes of one degree.  The coefficients are exact integers:
// each term coef * x (|x| <= p < 2^31: inputs are residues or the signed
// representatives in [-p, p) that intermediate launches store) is added to a
// signed 64-bit accumulator and
// the sum is reduced modulo p once per word (Sec. 3.5), in integer arithmetic
// only (modred.cuh).
//
// One launch processes a batch of independent tasks (factors of different
// strips); each block belongs to one task and covers 8 * RPW consecutive
// destination rows of it, one warp per row at a time.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "cp_internal.h"
#include "modred.cuh"

namespace cp {

__device__ __forceinline__ uint32_t reduce(long long acc, const ModRed &mr) {
    return modred_reduce(acc, mr.p, mr.m, mr.s);
}

__device__ __forceinline__ int edge_coef(uint32_t e, uint32_t sb) { return (int)e >> (sb + 2); }
__device__ __forceinline__ uint32_t edge_shift(uint32_t e, uint32_t sb) { return (e >> sb) & 3u; }
__device__ __forceinline__ uint32_t edge_src(uint32_t e, uint32_t sb) { return e & ((1u << sb) - 1u); }
__device__ __forceinline__ uint32_t fast_div(uint32_t x, uint32_t magic) { return magic ? __umulhi(x, magic) : x; }

constexpr int kWarps = kGatherThreads / 32;
constexpr unsigned kFull = 0xffffffffu;

// acc += coef * in[src][chunk c - shift*cpd], for the edges held one per lane
// in `my` (edge j in lane j), up to four loads in flight per lane.
template <bool V4>
__device__ __forceinline__ void gather_edges(const GatherTask &t, uint32_t my, int n, uint32_t c, uint32_t deg,
                                             bool active, long long *acc) {
    for (int e = 0; e < n; e += 4) {
        uint32_t q[4];
        uint4 x[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            q[j] = __shfl_sync(kFull, my, min(e + j, 31));
            const uint32_t sh = edge_shift(q[j], t.src_bits);
            x[j] = make_uint4(0, 0, 0, 0);
            if (e + j < n && active && deg >= sh) {
                const size_t off = (size_t)edge_src(q[j], t.src_bits) * t.C + (c - sh * t.cpd);
                if (V4) x[j] = __ldg(reinterpret_cast<const uint4 *>(t.in) + off);
                else x[j].x = __ldg(t.in + off);
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const long long cf = edge_coef(q[j], t.src_bits);  // absent edges loaded zero
            acc[0] += (long long)(int)x[j].x * cf;
            if (V4) {
                acc[1] += (long long)(int)x[j].y * cf;
                acc[2] += (long long)(int)x[j].z * cf;
                acc[3] += (long long)(int)x[j].w * cf;
            }
        }
    }
}

// One warp per destination row: the row's CSR entries are read once (two
// row_ptr words, then the edge list one edge per lane) and broadcast with
// shuffles; the lanes sweep the row's chunks 32 at a time.  The next row's
// CSR is fetched while the current row is computed.
template <int RPW, bool V4>
__device__ __forceinline__ void gather_rows(const GatherTask &t, uint32_t row0, const ModRed *s_mr) {
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t row = row0 + warp;
    uint32_t rp = (row < t.rows && lane < 2) ? __ldg(t.row_ptr + row + lane) : 0;
    uint32_t e0 = __shfl_sync(kFull, rp, 0), ne = __shfl_sync(kFull, rp, 1) - e0;
    uint32_t my = (row < t.rows && lane < ne) ? __ldg(t.edges + e0 + lane) : 0;
#pragma unroll 1
    for (int k = 0; k < RPW; ++k) {
        if (row >= t.rows) return;
        const uint32_t nrow = row + kWarps;
        uint32_t nrp = (k + 1 < RPW && nrow < t.rows && lane < 2) ? __ldg(t.row_ptr + nrow + lane) : 0;
#pragma unroll 1
        for (uint32_t j = t.c0; j < t.c0 + t.cw; j += 32) {
            const uint32_t c = j + lane;
            const bool active = c < t.c0 + t.cw;
            const uint32_t deg = fast_div(c, t.magic_cpd);
            const uint32_t pc = (c - deg * t.cpd) * (V4 ? 4 : 1);  // prime of the first word
            long long acc[4] = {modred_bias(s_mr[pc].p), V4 ? modred_bias(s_mr[pc + 1].p) : 0,
                                V4 ? modred_bias(s_mr[pc + 2].p) : 0, V4 ? modred_bias(s_mr[pc + 3].p) : 0};
            gather_edges<V4>(t, my, (int)min(ne, 32u), c, deg, active, acc);
            for (uint32_t eb = 32; eb < ne; eb += 32) {  // rows with more than 32 edges
                const uint32_t mb = (eb + lane < ne) ? __ldg(t.edges + e0 + eb + lane) : 0;
                gather_edges<V4>(t, mb, (int)min(ne - eb, 32u), c, deg, active, acc);
            }
            if (active) {
                const size_t o = (size_t)row * t.C + c;
                if (V4) {
                    const uint4 r = make_uint4(reduce(acc[0], s_mr[pc]), reduce(acc[1], s_mr[pc + 1]),
                                               reduce(acc[2], s_mr[pc + 2]), reduce(acc[3], s_mr[pc + 3]));
                    __stcs(reinterpret_cast<uint4 *>(t.out) + o, r);
                } else {
                    __stcs(t.out + o, reduce(acc[0], s_mr[pc]));
                }
            }
        }
        row = nrow;
        e0 = __shfl_sync(kFull, nrp, 0);
        ne = __shfl_sync(kFull, nrp, 1) - e0;
        my = (row < t.rows && lane < ne) ? __ldg(t.edges + e0 + lane) : 0;
    }
}

template <int RPW>
__global__ void __launch_bounds__(kGatherThreads) gather_kernel(const GatherTask *__restrict__ tasks, int n_tasks) {
    __shared__ ModRed s_mr[CP_MAX_PRIMES];
    // task of this block: the last one whose block_begin <= blockIdx.x (block-uniform)
    int lo = 0, hi = n_tasks - 1;
    const uint32_t b = blockIdx.x;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (tasks[mid].block_begin <= b) lo = mid; else hi = mid - 1;
    }
    const GatherTask t = tasks[lo];
    if (threadIdx.x < t.n_primes) {
        s_mr[threadIdx.x] = modred_make(__ldg(t.primes + threadIdx.x));
    }
    __syncthreads();
    // rows of the block: row0 + warp + 8 k, k < RPW
    const uint32_t row0 = (b - t.block_begin) * (uint32_t)(kWarps * RPW);
    if (t.vec4) gather_rows<RPW, true>(t, row0, s_mr);
    else gather_rows<RPW, false>(t, row0, s_mr);
}

bool tile_is_tma(int items) { return (items & 0xFFF) >= 16; }

uint32_t task_blocks(const GatherTask &t, int items) {
    const uint32_t per = tile_is_tma(items) ? (uint32_t)(items & 0xFFE) : (uint32_t)(kWarps * items);
    return (t.rows + per - 1) / per;
}

// For TMA tiles: chunks per thread (bits 24..27) default to 2 for rows wider
// than 3 KB (192 chunks), else 1; the block shape (bits 28..29) to narrow for
// rows of 129..160 chunks at one chunk per thread; edges per stage (bits
// 20..23) to about 20 KB of rows per stage (4 in narrow blocks); the ring
// (bits 12..19) to what fills the SM at the
// kernel's occupancy, raised to hold at least two stages of the widest row
// group.  A batch the TMA kernel cannot take uses the register kernel.
int effective_tile(const std::vector<GatherTask> &tasks, int items) {
    if (!tile_is_tma(items)) return items & 0xFFF;
    uint32_t max_rb = 0, max_cw = 0, min_cw = 0xffffffffu;
    for (auto &t : tasks) {
        if (!tma_usable(t)) return kGatherItems;
        max_rb = std::max(max_rb, t.cw * 16u);
        max_cw = std::max(max_cw, t.cw);
        min_cw = std::min(min_cw, t.cw);
    }
    int cpt = (items >> 24) & 15;
    if (cpt != 1 && cpt != 2 && cpt != 4) cpt = max_cw > 192 ? 2 : 1;
    // narrow blocks: 5 consumer warps cover rows of 129..160 chunks with at most
    // 31 idle lanes where the wide block leaves 3 of its 8 warps without a chunk
    const uint32_t cover = 32u * kTmaNarrowWarps;
    int shape = tile_shape(items);
    if (shape != 1 && shape != 2) shape = (cpt == 1 && min_cw > 128 && max_cw <= cover) ? 2 : 1;
    if (shape == 2 && (cpt != 1 || max_cw > cover)) shape = 1;
    uint32_t max_g = 1;
    if (shape == 1)
        for (auto &t : tasks) {
            uint32_t G = 1;  // row groups of the kernel's blocks (G * cw <= 256, at most one per consumer warp)
            while (G < 8u / (uint32_t)cpt && 2 * G * t.cw <= 256) G *= 2;
            max_g = std::max(max_g, G);
        }
    // (a narrow block has one row group)
    int edges = tile_edges(items);
    if (edges != 1 && edges != 2 && edges != 4 && edges != 8) {
        const uint32_t per = max_rb ? 20480u / max_rb : 8u;
        edges = per >= 8 ? 8 : (per >= 4 ? 4 : (per >= 2 ? 2 : 1));
        if (shape == 2) edges = 4;  // narrow blocks: six stages of 4 in the 52 KB ring beat three of 8
    }
    while ((uint32_t)edges * max_g > 32) edges /= 2;  // the producer warp has one lane per group and slot
    int ring = (items >> 12) & 0xFF;
    if (!ring) ring = tma_ring_kb_for(edges, cpt, shape == 2 ? kTmaNarrowWarps : 0);
    // a row group spans at most 4 KB of slot (G rows of cw chunks, G cw <= 256): two stages need 8 KB per edge
    ring = std::min(192, std::max(ring, std::max(16, 8 * edges)));
    return make_tile(items & 0xFFF, ring, edges, cpt) | (shape << 28);
}

// Rows per block of the default TMA tile: 32, or 16 where 32-row blocks would
// give a launch fewer than eight waves of resident blocks (about four per SM):
// on small strips the idle SMs of the last wave then cost more than the
// smaller blocks' set-up.
int default_rows(const std::vector<GatherTask> &tasks) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        sms = 152;
    uint64_t blocks = 0;
    for (auto &t : tasks) blocks += (t.rows + 31) / 32;
    return blocks >= 8ull * 4 * (uint64_t)sms ? 32 : 16;
}

uint32_t assign_blocks(std::vector<GatherTask> &tasks, int items) {
    uint32_t blk = 0;
    for (auto &t : tasks) {
        t.block_begin = blk;
        blk += task_blocks(t, items);
    }
    return blk;
}

// ceil(2^32 / d) for d >= 2 (0 encodes d == 1).
static uint32_t magic_for(uint32_t d) { return d <= 1 ? 0u : (uint32_t)(((1ull << 32) + d - 1) / d); }

void append_gather_tasks(std::vector<GatherTask> *tasks, const SiteTable &tab, const uint32_t *in, uint32_t *out,
                         const uint32_t *primes_dev, int D1, int P, bool partial) {
    const bool v4 = (P % 4) == 0;
    const uint32_t vec = v4 ? 4 : 1;
    GatherTask t{};
    t.in = in;
    t.out = out;
    t.row_ptr = tab.row_ptr;
    t.edges = tab.edges;
    t.primes = primes_dev;
    t.rows = (uint32_t)tab.n_dst;
    t.C = (uint32_t)((uint64_t)D1 * P / vec);
    t.cpd = (uint32_t)P / vec;
    t.vec4 = v4 ? 1 : 0;
    t.magic_cpd = magic_for(t.cpd);
    t.n_primes = (uint32_t)P;
    t.src_bits = (uint32_t)tab.op.src_bits;
    t.block_order = tab.block_order;
    t.partial = partial ? 1u : 0u;
    t.small_coefs = (tab.max_abs_coef <= kTmaMaxCoef && tab.max_coef_sum < kTmaMaxCoefSum) ? 1u : 0u;
    const uint32_t ncol = v4 ? (t.C + 255) / 256 : 1;
    for (uint32_t k = 0; k < ncol; ++k) {  // balanced column ranges
        t.c0 = (uint32_t)((uint64_t)t.C * k / ncol);
        t.cw = (uint32_t)((uint64_t)t.C * (k + 1) / ncol) - t.c0;
        tasks->push_back(t);
    }
}

int launch_gather_tma(const GatherTask *tasks_dev, int n_tasks, uint32_t total_blocks, int rpb, int *err,
                      cudaStream_t st, int edges, int ring_kb, int cpt, bool narrow);
int prepare_gather_tma();

int launch_gather(const GatherTask *tasks_dev, int n_tasks, uint32_t total_blocks, int items, cudaStream_t st) {
    if (n_tasks <= 0 || total_blocks == 0) return CP_OK;
    if (tile_is_tma(items))
        return launch_gather_tma(tasks_dev, n_tasks, total_blocks, items & 0xFFE, device_error_flag(), st,
                                 tile_edges(items), tile_ring_kb(items), tile_cpt(items), tile_shape(items) == 2);
    switch (items & 0xFFF) {
        case 1: gather_kernel<1><<<total_blocks, kGatherThreads, 0, st>>>(tasks_dev, n_tasks); break;
        case 2: gather_kernel<2><<<total_blocks, kGatherThreads, 0, st>>>(tasks_dev, n_tasks); break;
        case 4: gather_kernel<4><<<total_blocks, kGatherThreads, 0, st>>>(tasks_dev, n_tasks); break;
        case 8: gather_kernel<8><<<total_blocks, kGatherThreads, 0, st>>>(tasks_dev, n_tasks); break;
        default: return fail(CP_EINVAL, "gather tile must be 1, 2, 4, 8, 16, 32, 64 or 128");
    }
    CP_CUDA_TRY(cudaGetLastError());
    return CP_OK;
}

int prepare_gather_kernels() {
    int rc = prepare_gather_tma();
    if (rc) return rc;
    return device_error_flag() ? CP_OK : CP_ECUDA;
}

int *device_error_flag() {
    static int *flags[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    if (!flags[dev]) {
        int *p = nullptr;
        if (cudaMalloc(&p, sizeof(int)) != cudaSuccess) return nullptr;
        cudaMemset(p, 0, sizeof(int));
        cudaDeviceSynchronize();
        flags[dev] = p;
    }
    return flags[dev];
}

int check_device_error(cudaStream_t st) {
    int *f = device_error_flag();
    if (!f) return fail(CP_ECUDA, "device error word unavailable");
    CP_CUDA_TRY(cudaStreamSynchronize(st));
    int h = 0;
    CP_CUDA_TRY(cudaMemcpy(&h, f, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) {
        CP_CUDA_TRY(cudaMemset(f, 0, sizeof(int)));
        return fail(CP_ETIMEOUT, "a bounded wait in the TMA gather kernel ran out, or a block refused its "
                                 "configuration (flags " + std::to_string(h) + ")");
    }
    return CP_OK;
}

// [D1][P] -> [P][D1]
__global__ void transpose_row_kernel(const uint32_t *row, uint32_t *out, int D1, int P) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= D1 * P) return;
    int d = k / P, p = k - d * P;
    out[p * D1 + d] = row[k];
}

int launch_transpose_row(const uint32_t *row, uint32_t *out, int D1, int P, cudaStream_t st) {
    int n = D1 * P;
    transpose_row_kernel<<<(n + 255) / 256, 256, 0, st>>>(row, out, D1, P);
    CP_CUDA_TRY(cudaGetLastError());
    return CP_OK;
}

// Diagnostic: the gathers' reduction applied to given accumulator values.
__global__ void debug_reduce_kernel(const long long *v, const uint32_t *p, int n, uint32_t *out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const ModRed mr = modred_make(p[k]);
    out[k] = reduce(modred_bias(mr.p) + v[k], mr);
}

}  // namespace cp

extern "C" int cp_debug_reduce(const int64_t *v_host, const uint32_t *p_host, int n, uint32_t *out_host) {
    using namespace cp;
    if (n < 0 || (n > 0 && (!v_host || !p_host || !out_host))) return fail(CP_EINVAL, "bad arguments");
    for (int k = 0; k < n; ++k) {
        const uint32_t p = p_host[k];
        if (p < 2 || p >= (1u << 31)) return fail(CP_EINVAL, "p must be in [2, 2^31)");
        const long long lim = (long long)p * (long long)kReduceMaxCoefSum;
        if (v_host[k] <= -lim || v_host[k] >= lim) return fail(CP_EINVAL, "|v| must be below p * 2^20");
    }
    if (n == 0) return CP_OK;
    long long *v_d = nullptr;
    uint32_t *p_d = nullptr, *o_d = nullptr;
    int rc = dev_alloc((void **)&v_d, 8ull * n);
    if (!rc) rc = dev_alloc((void **)&p_d, 4ull * n);
    if (!rc) rc = dev_alloc((void **)&o_d, 4ull * n);
    cudaError_t e = cudaSuccess;
    if (!rc) {
        e = cudaMemcpy(v_d, v_host, 8ull * n, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(p_d, p_host, 4ull * n, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) {
            debug_reduce_kernel<<<(n + 255) / 256, 256>>>(v_d, p_d, n, o_d);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpy(out_host, o_d, 4ull * n, cudaMemcpyDeviceToHost);
    }
    dev_free(v_d);
    dev_free(p_d);
    dev_free(o_d);
    if (rc) return rc;
    if (e != cudaSuccess) return fail(CP_ECUDA, std::string("cp_debug_reduce: ") + cudaGetErrorString(e));
    return CP_OK;
}
