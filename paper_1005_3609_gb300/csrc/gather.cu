// The per-site operator kernel: one sparse factor T_i (or T_i^last) applied to
// a state vector, as a gather over the factor's CSR-by-destination table.
//
//   out[dst][d][p] = sum_{e in CSR(dst)} coef_e * in[src_e][d - shift_e][p]   (mod p)
//
// with in[..][d < 0] = 0 and degrees above D dropped: multiplying by w = 1/q
// is a shift of the coefficient index (Sec. 3.1, 3.5).  Rows are laid out
// [state][degree][prime], so a shift by one degree is a shift by n_primes
// words and, for n_primes % 4 == 0, every access is an aligned 16-byte load
// that reads four primes of one degree.  Arithmetic is add/sub mod p on
// 32-bit words with p < 2^31 (Sec. 3.5); no floating point.
//
// One launch processes a batch of independent tasks (factors of different
// strips); each block belongs to one task and covers 256 * ITEMS
// consecutive (dst, chunk) units of it.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "cp_internal.h"

namespace cp {

__device__ __forceinline__ uint32_t add_mod(uint32_t a, uint32_t b, uint32_t p) {
    uint32_t t = a + b - p;    // in (-p, p) as a signed value
    return min(t, t + p);      // unsigned min picks the representative in [0, p)
}

__device__ __forceinline__ uint32_t sub_mod(uint32_t a, uint32_t b, uint32_t p) {
    uint32_t t = a - b;
    return min(t, t + p);
}

// acc += coef * x (mod p) for the small coefficients that the factors produce.
__device__ __forceinline__ uint32_t axpy_mod(uint32_t acc, uint32_t x, int coef, uint32_t p) {
    if (coef > 0) {
        for (int k = 0; k < coef; ++k) acc = add_mod(acc, x, p);
    } else {
        for (int k = 0; k < -coef; ++k) acc = sub_mod(acc, x, p);
    }
    return acc;
}

__device__ __forceinline__ int edge_coef(uint32_t e) { return ((int)(e >> 29) << 29) >> 29; }
__device__ __forceinline__ uint32_t edge_shift(uint32_t e) { return (e >> kSrcBits) & 3u; }

template <int ITEMS>
__global__ void __launch_bounds__(kGatherThreads) gather_kernel(const GatherTask *__restrict__ tasks, int n_tasks) {
    // task of this block: the last one whose block_begin <= blockIdx.x
    int lo = 0, hi = n_tasks - 1;
    const uint32_t b = blockIdx.x;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (tasks[mid].block_begin <= b) lo = mid; else hi = mid - 1;
    }
    const GatherTask t = tasks[lo];
    const uint32_t base = (b - t.block_begin) * (uint32_t)(kGatherThreads * ITEMS);
#pragma unroll 1
    for (int it = 0; it < ITEMS; ++it) {
        const uint32_t u = base + it * kGatherThreads + threadIdx.x;
        if (u >= t.units) return;
        const uint32_t dst = u / t.C;
        const uint32_t c = u - dst * t.C;
        const uint32_t deg = c / t.cpd;
        const uint32_t pc = c - deg * t.cpd;
        const uint32_t e0 = __ldg(t.row_ptr + dst), e1 = __ldg(t.row_ptr + dst + 1);
        if (t.vec4) {
            const uint4 pr = __ldg(reinterpret_cast<const uint4 *>(t.primes) + pc);
            const uint4 *in = reinterpret_cast<const uint4 *>(t.in);
            uint32_t a0 = 0, a1 = 0, a2 = 0, a3 = 0;
            for (uint32_t e = e0; e < e1; ++e) {
                const uint32_t ed = __ldg(t.edges + e);
                const uint32_t sh = edge_shift(ed);
                if (deg < sh) continue;
                const int cf = edge_coef(ed);
                const uint4 x = __ldg(in + (size_t)(ed & kSrcMask) * t.C + (c - sh * t.cpd));
                a0 = axpy_mod(a0, x.x, cf, pr.x);
                a1 = axpy_mod(a1, x.y, cf, pr.y);
                a2 = axpy_mod(a2, x.z, cf, pr.z);
                a3 = axpy_mod(a3, x.w, cf, pr.w);
            }
            reinterpret_cast<uint4 *>(t.out)[(size_t)dst * t.C + c] = make_uint4(a0, a1, a2, a3);
        } else {
            const uint32_t p = __ldg(t.primes + pc);
            uint32_t a = 0;
            for (uint32_t e = e0; e < e1; ++e) {
                const uint32_t ed = __ldg(t.edges + e);
                const uint32_t sh = edge_shift(ed);
                if (deg < sh) continue;
                const uint32_t x = __ldg(t.in + (size_t)(ed & kSrcMask) * t.C + (c - sh * t.cpd));
                a = axpy_mod(a, x, edge_coef(ed), p);
            }
            t.out[(size_t)dst * t.C + c] = a;
        }
    }
}

uint32_t task_blocks(const GatherTask &t, int items) {
    const uint32_t per = (uint32_t)(kGatherThreads * items);
    return (t.units + per - 1) / per;
}

uint32_t assign_blocks(std::vector<GatherTask> &tasks, int items) {
    uint32_t blk = 0;
    for (auto &t : tasks) {
        t.block_begin = blk;
        blk += task_blocks(t, items);
    }
    return blk;
}

void append_gather_tasks(std::vector<GatherTask> *tasks, const SiteTable &tab, const uint32_t *in, uint32_t *out,
                         const uint32_t *primes_dev, int D1, int P) {
    const bool v4 = (P % 4) == 0;
    const uint32_t vec = v4 ? 4 : 1;
    const uint32_t C = (uint32_t)((uint64_t)D1 * P / vec);
    const uint32_t row_words = (uint32_t)D1 * P;
    const uint64_t max_rows = std::max<uint64_t>(1, (1ull << 31) / C);
    for (uint64_t r0 = 0; r0 < tab.n_dst; r0 += max_rows) {
        uint64_t nr = std::min<uint64_t>(max_rows, tab.n_dst - r0);
        GatherTask t{};
        t.in = in;
        t.out = out + r0 * row_words;
        t.row_ptr = tab.row_ptr + r0;
        t.edges = tab.edges;
        t.primes = primes_dev;
        t.units = (uint32_t)(nr * C);
        t.C = C;
        t.cpd = (uint32_t)P / vec;
        t.vec4 = v4 ? 1 : 0;
        tasks->push_back(t);
    }
}

int launch_gather(const GatherTask *tasks_dev, int n_tasks, uint32_t total_blocks, int items, cudaStream_t st) {
    if (n_tasks <= 0 || total_blocks == 0) return CP_OK;
    switch (items) {
        case 1: gather_kernel<1><<<total_blocks, kGatherThreads, 0, st>>>(tasks_dev, n_tasks); break;
        case 2: gather_kernel<2><<<total_blocks, kGatherThreads, 0, st>>>(tasks_dev, n_tasks); break;
        case 4: gather_kernel<4><<<total_blocks, kGatherThreads, 0, st>>>(tasks_dev, n_tasks); break;
        case 8: gather_kernel<8><<<total_blocks, kGatherThreads, 0, st>>>(tasks_dev, n_tasks); break;
        default: return fail(CP_EINVAL, "gather tile must be 1, 2, 4 or 8");
    }
    CP_CUDA_TRY(cudaGetLastError());
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

}  // namespace cp
