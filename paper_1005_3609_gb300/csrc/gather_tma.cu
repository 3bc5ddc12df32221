// The per-site gather with TMA bulk copies (rows of 16-byte chunks only).
//
// Same operation as gather_kernel: out[dst] = sum_e coef_e w^{shift_e} in[src_e]
// (mod p).  A block owns a range of destination rows of one task.  Warp 0 is
// the producer: it walks the block's CSR edges in order, a few at a time with
// one lane per edge, and for each edge copies the part of the source row that
// survives the shift by w^{shift}
// (degrees 0 .. D-shift) with one cp.async.bulk into the next slot of a
// shared-memory ring, placed at degree offset `shift`, so that slot chunk c is
// the source value that destination chunk c needs.  Each slot has a "full"
// mbarrier (completed by the copy's byte count) and an "empty" mbarrier
// (completed when the eight consumer warps are done with it).  Warps 1..8
// consume the slots in the same order: coef * slot[c] into signed 64-bit
// accumulators, one reduction mod p per word, streaming stores of the
// destination row.  With a 28 KB ring, seven blocks share an SM (seven
// producers, ~196 KB of source rows in flight per SM) without using registers.
//
// Every mbarrier wait is bounded (kWaitCycles); on expiry the thread sets
// *err and returns, and the producer first waits (bounded) for the copies it
// has issued to land.  Blocks that start after an error return at once.
#include <cuda_runtime.h>

#include <string>

#include "cp_internal.h"

namespace cp {

constexpr int kTmaConsumers = 8;                      // consumer warps
constexpr int kTmaThreads = 32 * (kTmaConsumers + 1);  // + producer warp
constexpr int kTmaMaxSlots = 96;
constexpr int kTmaMaxPasses = 8;                       // C <= 8 * 256 chunks
// Copies the producer warp issues together: about kIssueBytes per batch, at
// least 2 and at most kIssueBatchMax (narrow rows need more copies in flight).
constexpr uint32_t kIssueBytes = 8192;
constexpr uint32_t kIssueBatchMax = 16;
constexpr long long kWaitCycles = 1ll << 31;           // ~1 s at 2 GHz

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t a, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
// The suspend-time hint (ns) lets a waiting warp sleep in the barrier instead of
// re-issuing the test: the gather is bound by instruction issue on the SMs, and
// polling warps took issue slots from the working ones (about 1% of the time).
constexpr uint32_t kWaitHintNs = 20000;

__device__ __forceinline__ bool mbar_try_wait(uint32_t a, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity), "r"(kWaitHintNs)
        : "memory");
    return ok != 0;
}
// Wait for the phase of parity `parity` to complete; false once the deadline passes.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, long long deadline) {
    while (!mbar_try_wait(a, parity))
        if (clock64() > deadline) return false;
    return true;
}
__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}

__device__ __forceinline__ uint32_t fast_div_u(uint32_t x, uint32_t magic) { return magic ? __umulhi(x, magic) : x; }

// v mod p for |v| < p * sum|coef| <= p * 2^20 (the table build enforces the
// bound).  The quotient estimate fl(fl(v) * fl(1/p) - 1/2), fused, is within
// 1/4 of v/p - 1/2 (relative error of the product < 3 * 2^-24 on |v/p| < 2^20,
// plus half an ulp below 2^20), so its floor q' gives v - q' p in (p/4, 7p/4),
// below 2^32 for p < 2^31, and one conditional subtraction finishes.
__device__ __forceinline__ uint32_t reduce_s64_t(long long v, uint32_t p, float invp) {
    const int q = __float2int_rd(__fmaf_rn(__ll2float_rn(v), invp, -0.5f));
    const uint32_t r = (uint32_t)v - (uint32_t)q * p;
    return min(r, r - p);
}

// Consumer mapping: the 8 consumer warps form G row groups (G a power of two,
// the largest <= 8 with ceil(C G / 256) <= PASSES).  Group g (warps
// 1 + (8/G) g .. (8/G)(g+1)) handles the rows r = g (mod G) of the block; its
// 256/G threads cover a row's C chunks, up to PASSES chunks per thread.  Each
// group has its own sub-ring of slots, filled by the producer and consumed by
// the group strictly in order (a group never runs ahead of the slot phases it
// waits on).  More chunks per thread spread the per-edge work (barrier wait,
// edge decode, release) over more data and put G rows in flight per block.
template <int RPB, int PASSES>
__global__ void __launch_bounds__(kTmaThreads, PASSES == 1 ? 7 : (PASSES == 2 ? 3 : (PASSES == 4 ? 2 : 1)))
    gather_tma_kernel(const GatherTask *__restrict__ tasks, int n_tasks, uint32_t ring_bytes, int *err) {
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ uint64_t full_bar[kTmaMaxSlots], empty_bar[kTmaMaxSlots];
    __shared__ uint32_t meta[kTmaMaxSlots];
    __shared__ uint32_t s_rp[RPB + 1];
    __shared__ uint32_t s_gpos[RPB];  // first sub-ring position of each row's edges
    __shared__ uint32_t s_gtot[8];    // edges per sub-ring
    __shared__ uint32_t s_p[CP_MAX_PRIMES];
    __shared__ float s_inv[CP_MAX_PRIMES];
    __shared__ int s_abort;

    if (threadIdx.x == 0) s_abort = *(volatile int *)err;  // a previous block gave up: do nothing
    __syncthreads();
    if (s_abort) return;
    int lo = 0, hi = n_tasks - 1;
    const uint32_t b = blockIdx.x;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (tasks[mid].block_begin <= b) lo = mid; else hi = mid - 1;
    }
    const GatherTask t = tasks[lo];
    const uint32_t row0 = (b - t.block_begin) * (uint32_t)RPB;
    const uint32_t nrows = min((uint32_t)RPB, t.rows - row0);
    // a slot holds the column range [c0, c0 + cw) of a row: slot chunk x is
    // source chunk c0 + x - shift * cpd (absent where that is negative)
    const uint32_t RB = t.cw * 16u;                             // slot bytes
    const uint8_t *in_bytes = reinterpret_cast<const uint8_t *>(t.in);
    const size_t src_row_bytes = (size_t)t.C * 16u;
    uint32_t G = 1;
    while (G < 8 && (t.cw * 2 * G + 255) / 256 <= (uint32_t)PASSES) G *= 2;
    // G sub-rings of nsub slots each; slot of sub-ring position x = x mod nsub, phase = (x / nsub) & 1
    uint32_t nsub = min((uint32_t)kTmaMaxSlots / G, ring_bytes / (G * RB));
    if (nsub == 0) {  // ring smaller than one row per group: refuse (block-uniform)
        if (threadIdx.x == 0) atomicOr(err, 8);
        return;
    }
    const uint32_t nmagic = nsub > 1 ? (uint32_t)(((1ull << 32) + nsub - 1) / nsub) : 0u;  // exact for x * nsub < 2^32
    const uint32_t nslot = G * nsub;

    for (uint32_t i = threadIdx.x; i <= nrows; i += blockDim.x) s_rp[i] = __ldg(t.row_ptr + row0 + i);
    if (threadIdx.x < t.n_primes) {
        const uint32_t p = __ldg(t.primes + threadIdx.x);
        s_p[threadIdx.x] = p;
        s_inv[threadIdx.x] = 1.0f / (float)p;
    }
    if (threadIdx.x == 0) {
        for (uint32_t s = 0; s < nslot; ++s) {
            mbar_init(smem_addr(&full_bar[s]), 1);
            mbar_init(smem_addr(&empty_bar[s]), kTmaConsumers / G);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (G > 1 && threadIdx.x < G) {  // positions of each row's edges within its sub-ring
        uint32_t run = 0;
        for (uint32_t r = threadIdx.x; r < nrows; r += G) {
            s_gpos[r] = run;
            run += s_rp[r + 1] - s_rp[r];
        }
        s_gtot[threadIdx.x] = run;
    }
    if (G == 1 && threadIdx.x == 0) s_gtot[0] = s_rp[nrows] - s_rp[0];
    __syncthreads();
    const long long deadline = clock64() + kWaitCycles;
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (warp == 0) {
        // ---------------- producer: one bulk copy per edge, in CSR order, the
        // copies of B consecutive edges issued together, one lane per edge
        // (B <= nsub: a batch holds at most nsub edges of any sub-ring, so its slots
        // are distinct); a lane finds its edge's row by binary search of the
        // block's row pointers, hence the edge's sub-ring and position in it.
        // Issuing from several lanes keeps more copies in flight than one lane
        // walking the edges could.
        const uint32_t e_begin = s_rp[0], e_end = s_rp[nrows];
        const uint32_t B = min(nsub, min(kIssueBatchMax, max(2u, kIssueBytes / RB)));
        bool ok = true;
        uint32_t qn = (lane < B && e_begin + lane < e_end) ? __ldg(t.edges + e_begin + lane) : 0u;
        for (uint32_t base = e_begin; base < e_end && ok; base += B) {
            const uint32_t e = base + lane;
            const uint32_t qj = qn;
            qn = (lane < B && e + B < e_end) ? __ldg(t.edges + e + B) : 0u;  // next batch
            bool lok = true;
            if (lane < B && e < e_end) {
                uint32_t g = 0, cnt = e - e_begin;
                if (G > 1) {  // row of the edge: the last r with s_rp[r] <= e
                    uint32_t lo = 0, hi = nrows - 1;
                    while (lo < hi) {
                        const uint32_t mid = (lo + hi + 1) >> 1;
                        if (s_rp[mid] <= e) lo = mid; else hi = mid - 1;
                    }
                    g = lo & (G - 1);
                    cnt = s_gpos[lo] + (e - s_rp[lo]);
                }
                const uint32_t qd = fast_div_u(cnt, nmagic);
                const uint32_t s = g * nsub + (cnt - qd * nsub), ph = qd & 1u;
                if (cnt >= nsub && !mbar_wait(smem_addr(&empty_bar[s]), ph ^ 1u, deadline)) {
                    atomicOr(err, 2);
                    lok = false;
                }
                if (lok) {
                    meta[s] = qj;
                    const uint32_t back = ((qj >> t.src_bits) & 3u) * t.cpd;  // shift in chunks
                    const uint32_t skip = back > t.c0 ? min(back - t.c0, t.cw) : 0u;
                    const uint32_t bytes = (t.cw - skip) * 16u;
                    const uint32_t fb = smem_addr(&full_bar[s]);
                    if (bytes) {
                        mbar_arrive_expect_tx(fb, bytes);
                        bulk_copy_g2s(smem_addr(smem + (size_t)s * RB + skip * 16u),
                                      in_bytes + (size_t)(qj & ((1u << t.src_bits) - 1u)) * src_row_bytes +
                                          (size_t)(t.c0 + skip - back) * 16u,
                                      bytes, fb);
                    } else {
                        mbar_arrive(fb);
                    }
                }
            }
            ok = __all_sync(0xffffffffu, lok);
        }
        // do not leave while own copies are in flight: wait for the last ones of every sub-ring
        if (lane == 0) {
            for (uint32_t g = 0; g < G; ++g) {
                const uint32_t cnt = s_gtot[g], last = min(cnt, nsub);
                for (uint32_t k = 0; k < last; ++k) {
                    const uint32_t i = cnt - 1 - k, qd = fast_div_u(i, nmagic);
                    if (!mbar_wait(smem_addr(&full_bar[g * nsub + (i - qd * nsub)]), qd & 1u,
                                   deadline + kWaitCycles)) {
                        atomicOr(err, 4);
                        g = G;
                        break;
                    }
                }
            }
        }
        return;
    }

    // ---------------- consumers
    const uint32_t cw = warp - 1;                   // consumer warp 0..7
    const uint32_t grp = cw / (kTmaConsumers / G);  // row group = sub-ring
    const uint32_t GT = 256 / G;                    // threads per group
    const uint32_t gt = threadIdx.x - 32 - grp * GT;  // thread within the group
    uint32_t deg[PASSES];
#pragma unroll
    for (int p = 0; p < PASSES; ++p) deg[p] = fast_div_u(t.c0 + gt + GT * p, t.magic_cpd);
    const int passes = (int)((t.cw + GT - 1) / GT);
    uint32_t slot = 0, phase = 0;  // next slot of this sub-ring and its phase parity
    for (uint32_t r = grp; r < nrows; r += G) {
        const uint32_t ne = s_rp[r + 1] - s_rp[r];
        long long acc[PASSES][4];
#pragma unroll
        for (int p = 0; p < PASSES; ++p) acc[p][0] = acc[p][1] = acc[p][2] = acc[p][3] = 0;
        for (uint32_t j = 0; j < ne; ++j) {
            const uint32_t s = grp * nsub + slot;
            if (!mbar_wait(smem_addr(&full_bar[s]), phase, deadline)) {
                atomicOr(err, 1);
                return;
            }
            const uint32_t q = meta[s];
            const uint32_t sh = (q >> t.src_bits) & 3u;
            const long long cf = (int)q >> (t.src_bits + 2);
            const uint4 *sd = reinterpret_cast<const uint4 *>(smem + (size_t)s * RB);
#pragma unroll
            for (int p = 0; p < PASSES; ++p) {
                const uint32_t c = gt + GT * p;  // chunk within the column range
                if (p < passes && c < t.cw && deg[p] >= sh) {
                    const uint4 x = sd[c];
                    acc[p][0] += (long long)(int)x.x * cf;
                    acc[p][1] += (long long)(int)x.y * cf;
                    acc[p][2] += (long long)(int)x.z * cf;
                    acc[p][3] += (long long)(int)x.w * cf;
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_addr(&empty_bar[s]));
            if (++slot == nsub) {
                slot = 0;
                phase ^= 1u;
            }
        }
        const size_t orow = (size_t)(row0 + r) * t.C + t.c0;
#pragma unroll
        for (int p = 0; p < PASSES; ++p) {
            const uint32_t c = gt + GT * p;
            if (p < passes && c < t.cw) {
                const uint32_t pc = (t.c0 + c - deg[p] * t.cpd) * 4;
                const uint4 v = make_uint4(reduce_s64_t(acc[p][0], s_p[pc], s_inv[pc]),
                                           reduce_s64_t(acc[p][1], s_p[pc + 1], s_inv[pc + 1]),
                                           reduce_s64_t(acc[p][2], s_p[pc + 2], s_inv[pc + 2]),
                                           reduce_s64_t(acc[p][3], s_p[pc + 3], s_inv[pc + 3]));
                __stcs(reinterpret_cast<uint4 *>(t.out) + orow + c, v);
            }
        }
    }
}

// Ring sizes: one chunk pass uses ring_kb KB (several blocks per SM), more
// passes the largest ring (one block per SM).
constexpr uint32_t kTmaRingMax = 192 * 1024;
constexpr uint32_t kTmaRingMin = 16 * 1024;

bool tma_usable(const GatherTask &t) {
    if (!t.vec4 || t.cw > (uint32_t)(256 * kTmaMaxPasses)) return false;
    return kTmaRingMax / (t.cw * 16u) >= 8;
}

template <int RPB, int PASSES>
static int set_attr() {
    const int dyn = (int)kTmaRingMax;
    CP_CUDA_TRY(cudaFuncSetAttribute(gather_tma_kernel<RPB, PASSES>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn));
    return CP_OK;
}

template <int PASSES>
static int set_attrs() {
    int rc;
    if ((rc = set_attr<16, PASSES>()) || (rc = set_attr<32, PASSES>()) || (rc = set_attr<64, PASSES>()) ||
        (rc = set_attr<128, PASSES>()))
        return rc;
    return CP_OK;
}

// Diagnostic: a wait that can never complete (an mbarrier nothing arrives on),
// bounded by `cycles`; on expiry it sets bit 16 of *err and returns, like the
// gather kernels' waits.
__global__ void wait_timeout_kernel(long long cycles, int *err) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) mbar_init(smem_addr(&bar), 1);
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait(smem_addr(&bar), 0, clock64() + cycles)) atomicOr(err, 1 << 16);
}

int debug_wait_timeout(long long cycles, cudaStream_t st) {
    wait_timeout_kernel<<<1, 32, 0, st>>>(cycles, device_error_flag());
    CP_CUDA_TRY(cudaGetLastError());
    return check_device_error(st);
}

int prepare_gather_tma() {
    static bool done[64] = {};
    int dev = 0;
    CP_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(CP_EINVAL, "device index");
    if (done[dev]) return CP_OK;
    int rc;
    if ((rc = set_attrs<1>()) || (rc = set_attrs<2>()) || (rc = set_attrs<4>()) || (rc = set_attrs<8>())) return rc;
    done[dev] = true;
    return CP_OK;
}

template <int PASSES>
static void launch_passes(int rpb, const GatherTask *tasks_dev, int n_tasks, uint32_t blocks, uint32_t dyn, int *err,
                          cudaStream_t st) {
    switch (rpb) {
        case 16: gather_tma_kernel<16, PASSES><<<blocks, kTmaThreads, dyn, st>>>(tasks_dev, n_tasks, dyn, err); break;
        case 32: gather_tma_kernel<32, PASSES><<<blocks, kTmaThreads, dyn, st>>>(tasks_dev, n_tasks, dyn, err); break;
        case 64: gather_tma_kernel<64, PASSES><<<blocks, kTmaThreads, dyn, st>>>(tasks_dev, n_tasks, dyn, err); break;
        default: gather_tma_kernel<128, PASSES><<<blocks, kTmaThreads, dyn, st>>>(tasks_dev, n_tasks, dyn, err); break;
    }
}

// passes: chunks per consumer thread (1, 2, 4 or 8); every task must have C <= 256 * passes.
int launch_gather_tma(const GatherTask *tasks_dev, int n_tasks, uint32_t total_blocks, int rpb, int *err,
                      cudaStream_t st, int passes, int ring_kb) {
    if (n_tasks <= 0 || total_blocks == 0) return CP_OK;
    if (rpb != 16 && rpb != 32 && rpb != 64 && rpb != 128)
        return fail(CP_EINVAL, "TMA gather rows per block must be 16, 32, 64 or 128");
    uint32_t dyn = (uint32_t)ring_kb * 1024u;
    if (dyn < kTmaRingMin) dyn = kTmaRingMin;
    if (dyn > kTmaRingMax) dyn = kTmaRingMax;
    if (passes == 1) launch_passes<1>(rpb, tasks_dev, n_tasks, total_blocks, dyn, err, st);
    else if (passes == 2) launch_passes<2>(rpb, tasks_dev, n_tasks, total_blocks, dyn, err, st);
    else if (passes == 4) launch_passes<4>(rpb, tasks_dev, n_tasks, total_blocks, dyn, err, st);
    else launch_passes<8>(rpb, tasks_dev, n_tasks, total_blocks, dyn, err, st);
    CP_CUDA_TRY(cudaGetLastError());
    return CP_OK;
}

}  // namespace cp
