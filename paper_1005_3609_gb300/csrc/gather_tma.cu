// The per-site gather with TMA bulk copies (rows of 16-byte chunks only).
//
// Same operation as gather_kernel: out[dst] = sum_e coef_e w^{shift_e} in[src_e]
// (mod p), one per-site factor of Sec. 3.2-3.3 (multiplication by w a shift of
// the degree index).  A block owns a range of destination rows of one task and
// splits it into G row groups (G the largest power of two <= 8 with G times the
// task's row chunks <= 256), each a contiguous run of rows, so that every group
// consumes one contiguous run of CSR edges.
//
// Warp 0 is the producer.  For each group it walks the group's edges in CSR
// order, E at a time (a "stage"), one lane per edge: the lane copies the part
// of the edge's source row that survives the shift by w^shift with one
// cp.async.bulk into its slot of the stage, placed at degree offset `shift` (so
// slot chunk c is the source value destination chunk c needs), and records the
// edge's coefficient and shift beside the slot.  A stage has one "full"
// mbarrier (E arrivals, completed with the copies' byte count) and one "empty"
// mbarrier (one arrival per consumer warp of the group): consumers wait once
// per stage, not once per edge.
//
// Warps 1..W are the consumers, W/G per group, CPT 16-byte chunks (four primes
// of one degree each) per thread: W = 8 / CPT (a wide block, 256 chunks), or
// W = 5 at CPT 1 (a narrow block for rows of 129..160 chunks, one group);
// warps whose chunks all lie beyond the row leave at once.  Per stage a
// consumer reads the E coefficients, then edge by edge its chunks of the slots,
// adding coef * chunk into pairs of 32-bit sums (two 16 x 8-bit dot products
// per word; tables with |coef| > 127 or coefficient sums of 2^15 and more use
// the register kernel), and releases the stage;
// when the CSR reaches the end of a destination row the thread reduces its four
// words modulo their primes (integer Barrett, modred.cuh) and streams them out.
//
// Every mbarrier wait is bounded (kWaitCycles); on expiry the thread sets *err
// and returns, and the producer first waits (bounded) for the copies it has
// issued to land.  Blocks that start after an error return at once.
#include <cuda_runtime.h>

#include <string>

#include "cp_internal.h"
#include "modred.cuh"

namespace cp {

constexpr int kTmaConsumers = 8;                      // consumer warps at one chunk per thread
constexpr int kTmaMaxSlots = 96;                       // row slots per block (all groups)
constexpr int kTmaMaxRows = 128;                       // destination rows per block
constexpr int kTmaMaxShift = 3;                        // shifts of the edge format: 2 bits
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
// re-issuing the test, leaving the issue slots to the warps that have work.
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

// Shared state of one block.
struct TmaShared {
    uint64_t full_bar[kTmaMaxSlots], empty_bar[kTmaMaxSlots];  // per stage (at most one stage per slot)
    alignas(16) int cf[kTmaMaxSlots];       // per slot: the edge's coefficient
    alignas(16) uint32_t sh[kTmaMaxSlots];  // per slot: the edge's shift (degrees)
    alignas(16) uint32_t p[CP_MAX_PRIMES];  // reduction constants per prime
    alignas(16) uint32_t m[CP_MAX_PRIMES];
    alignas(16) uint32_t s[CP_MAX_PRIMES];
    alignas(16) uint32_t l0[CP_MAX_PRIMES];  // start of a word's sums: lo = (p & 1) 2^15, hi = p >> 1,
    alignas(16) uint32_t h0[CP_MAX_PRIMES];  // so that hi 2^16 + lo starts at B = p 2^15
    uint32_t rp[kTmaMaxRows + 1];           // the block's row pointers
    long long deadline;            // clock64 limit of every wait
    GatherTask task;               // the block's task (read where needed, not held in registers)
    int abort_flag;
};

// Geometry of one block, identical in every thread.
struct TmaBlock {
    uint32_t row0, nrows, G, NS, act;
};

__device__ __forceinline__ void tma_group_rows(const TmaBlock &bk, uint32_t g, uint32_t *r0, uint32_t *r1) {
    *r0 = bk.nrows * g / bk.G;
    *r1 = bk.nrows * (g + 1) / bk.G;
}

// ---------------------------------------------------------------- producer
// Stages of a group: its edges in CSR order, E per stage (the last stage of the
// group may be partly empty: coefficient 0, no copy).  Stages are not aligned
// to destination rows; the consumers find the row ends from the row pointers.
template <int E>
__device__ __forceinline__ void tma_produce(const GatherTask &t, const TmaBlock &bk, TmaShared &S, uint8_t *ring,
                                            int *err) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t g = lane / E, j = lane - g * E;  // lane j of group g's stages (G * E <= 32)
    const bool has = g < bk.G;
    uint32_t r0 = 0, r1 = 0, gb = 0, gn = 0;
    if (has) {
        tma_group_rows(bk, g, &r0, &r1);
        gb = S.rp[r0];
        gn = S.rp[r1] - gb;
    }
    const uint32_t kmax = __reduce_max_sync(0xffffffffu, has ? (gn + E - 1) / E : 0u);
    const uint32_t RB = t.cw * 16u;
    const uint8_t *in_bytes = reinterpret_cast<const uint8_t *>(t.in);
    const size_t src_row_bytes = (size_t)t.C * 16u;
    const uint32_t src_mask = (1u << t.src_bits) - 1u;
    const long long deadline = S.deadline;
    uint32_t q = (has && j < gn) ? __ldg(t.edges + gb + j) : 0u;
    uint32_t s = 0, ph = 0;
    for (uint32_t k = 0; k < kmax; ++k) {
        const uint32_t idx = k * E + j;  // edge within the group
        const uint32_t qn = (has && idx + E < gn) ? __ldg(t.edges + gb + idx + E) : 0u;  // next stage's edge
        bool lok = true;
        if (has && k * E < gn) {  // the group has a stage k
            const uint32_t st = g * bk.NS + s;
            if (k >= bk.NS && !mbar_wait(smem_addr(&S.empty_bar[st]), ph ^ 1u, deadline)) {
                atomicOr(err, 2);
                lok = false;
            }
            if (lok) {
                const uint32_t fb = smem_addr(&S.full_bar[st]);
                const uint32_t slot = st * E + j;
                if (idx < gn) {
                    const uint32_t sh = (q >> t.src_bits) & 3u;
                    const uint32_t cb = (uint32_t)((int)q >> (t.src_bits + 2)) & 0xFFu;
                    S.cf[slot] = (int)(cb | (cb << 24));  // coefficient in bytes 0 and 3 (see mad_dp2a)
                    S.sh[slot] = sh;
                    const uint32_t back = sh * t.cpd;  // shift in chunks
                    const uint32_t skip = back > t.c0 ? min(back - t.c0, t.cw) : 0u;
                    const uint32_t bytes = (t.cw - skip) * 16u;
                    if (bytes) {
                        mbar_arrive_expect_tx(fb, bytes);
                        bulk_copy_g2s(smem_addr(ring + (size_t)slot * RB + skip * 16u),
                                      in_bytes + (size_t)(q & src_mask) * src_row_bytes +
                                          (size_t)(t.c0 + skip - back) * 16u,
                                      bytes, fb);
                    } else {
                        mbar_arrive(fb);
                    }
                } else {  // past the group's last edge: a slot that adds nothing
                    S.cf[slot] = 0;
                    S.sh[slot] = 0;
                    mbar_arrive(fb);
                }
            }
        }
        if (!__all_sync(0xffffffffu, lok)) break;
        q = qn;
        if (++s == bk.NS) {
            s = 0;
            ph ^= 1u;
        }
    }
    // do not leave while own copies are in flight: one lane per group waits
    // (bounded) for the group's last NS stages to have landed
    if (has && j == 0) {
        const uint32_t kg = (gn + E - 1) / E;
        const uint32_t last = min(kg, bk.NS);
        for (uint32_t i = 0; i < last; ++i) {
            const uint32_t k = kg - 1 - i;
            if (!mbar_wait(smem_addr(&S.full_bar[g * bk.NS + k % bk.NS]), (k / bk.NS) & 1u, deadline + kWaitCycles)) {
                atomicOr(err, 4);
                return;
            }
        }
    }
}

// 16-byte shared load, executed only where pred != 0 (zero elsewhere), with
// the predicate inside the instruction so that the warp does not branch.
__device__ __forceinline__ uint4 lds128_if(uint32_t addr, uint32_t pred) {
    uint4 v = make_uint4(0, 0, 0, 0);
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %5, 0;\n\t"
        "@p ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];\n\t}"
        : "+r"(v.x), "+r"(v.y), "+r"(v.z), "+r"(v.w)
        : "r"(addr), "r"(pred));
    return v;
}
__device__ __forceinline__ uint4 lds128(uint32_t addr) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(addr));
    return v;
}
// Exact sums without 64-bit multiply-adds.  An input word x (a residue in
// [0, p) or a signed representative in [-p, p), as 32-bit two's complement)
// is x = xh 2^16 + xl with xl = x & 0xffff (unsigned) and xh = x >> 16
// (signed).  The edge's coefficient c (|c| <= 127) sits in bytes 0 and 3 of b,
// so dp2a.lo (x's halves times b's bytes 0, 1) adds c xl and dp2a.hi (times
// bytes 2, 3) adds c xh, each into a 32-bit sum: with S = sum |c| < 2^15 over
// the destination's edges and the starting values below (lo <= 2^15, hi <
// 2^30), |lo| <= 2^15 + S (2^16 - 1) < 2^31 and |hi| < 2^30 + S 2^15 < 2^31,
// and hi 2^16 + lo is the start plus sum_e c_e x_e, exactly.  Two 32-bit
// instructions per word and edge where a widening 64-bit multiply-add costs
// about three.
struct Acc2 {
    int lo, hi;
};
__device__ __forceinline__ void mad_dp2a(Acc2 &acc, uint32_t x, int b) {
    asm("dp2a.lo.u32.s32 %0, %2, %3, %0;\n\tdp2a.hi.s32.s32 %1, %2, %3, %1;"
        : "+r"(acc.lo), "+r"(acc.hi)
        : "r"(x), "r"(b));
}
// The sums start at B = p 2^15 (a multiple of p above |sum_e c_e x_e| <= S p),
// so u = hi 2^16 + lo = B + sum_e c_e x_e lies in (0, p 2^16).
//
// u mod p for primes p >= 2^17 in 32-bit arithmetic: the quotient estimate of
// modred.cuh with s = b - 2 >= 16 takes h = floor(u / 2^s) = floor((hi +
// floor(lo / 2^16)) / 2^(s-16)) (c = s - 16); as u < 2^(b+16) the error terms
// stay below 2^-14 + 1/2, so r = u - q p (taken modulo 2^32, with u's low word
// hi 2^16 + lo) lies in [0, 2p).  Returns r reduced (full) or r - p.
__device__ __forceinline__ uint32_t reduce_halves(const Acc2 &a, uint32_t p, uint32_t m, uint32_t c, bool full) {
    const uint32_t h = (uint32_t)(a.hi + (a.lo >> 16)) >> c;
    const uint32_t q = __umulhi(h, m);
    const uint32_t r = ((uint32_t)a.hi << 16) + (uint32_t)a.lo - q * p;
    return full ? min(r, r - p) : r - p;
}
// Any prime: p 2^21 + u as the accumulator of modred.cuh.
__device__ __forceinline__ long long acc_value(const Acc2 &a, uint32_t p) {
    return modred_bias(p) + ((long long)a.hi << 16) + a.lo;
}
// Arrive on an mbarrier from the lanes where pred != 0, without branching.
__device__ __forceinline__ void mbar_arrive_if(uint32_t a, uint32_t pred) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %1, 0;\n\t"
        "@p mbarrier.arrive.shared::cta.b64 _, [%0];\n\t}" ::"r"(a), "r"(pred)
        : "memory");
}
// Streaming 16-byte global store where pred != 0.
__device__ __forceinline__ void stcs128_if(uint4 *ptr, uint4 v, uint32_t pred) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %5, 0;\n\t"
        "@p st.global.cs.v4.u32 [%0], {%1, %2, %3, %4};\n\t}" ::"l"(ptr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w),
        "r"(pred)
        : "memory");
}

// ---------------------------------------------------------------- consumers
// A consumer thread owns CPT chunks of the row, c + k * stride (stride = the
// chunks its group's warps cover side by side), so a warp's 16-byte loads
// stay contiguous.  Per stage: the E coefficients, then edge by edge the
// thread's chunks and their multiply-adds; after the last edge of a row (and
// for the empty rows that follow it) reduce the words and store them; then
// release the stage.  Chunks past the row's end are read from a valid chunk
// and not stored.  PRED: the warp holds chunks of degree < kTmaMaxShift (only
// the first chunk can), where a shifted copy leaves the slot's low chunks
// unwritten and the shift must be checked.
template <int E, int CPT, bool PRED, bool FULL, bool FR>
__device__ __forceinline__ void tma_consume(const GatherTask &t, const TmaBlock &bk, TmaShared &S, uint32_t ring_addr,
                                            uint32_t g, uint32_t c, uint32_t stride, int *err) {
    const uint32_t lane = threadIdx.x & 31;
    uint32_t col[CPT], gcs[CPT], pcs[CPT], active[CPT];
    uint32_t deg0 = 0;
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
        const uint32_t ck = c + k * stride;
        active[k] = ck < t.cw ? 1u : 0u;
        const uint32_t cl = min(ck, t.cw - 1);  // the chunk this thread reads
        gcs[k] = t.c0 + cl;                      // chunk within the row
        const uint32_t deg = fast_div_u(gcs[k], t.magic_cpd);
        if (k == 0) deg0 = deg;
        pcs[k] = (gcs[k] - deg * t.cpd) * 4u;  // prime of the chunk's first word (a multiple of 4)
        col[k] = ring_addr + cl * 16u;
    }
    // reduction constants of the first chunk's four primes, kept in registers; the other
    // chunks have the same primes when the stride is a multiple of the chunks per degree
    const bool same_primes = stride % t.cpd == 0;
    const uint4 P0 = *reinterpret_cast<const uint4 *>(S.p + pcs[0]);
    const uint4 M0 = *reinterpret_cast<const uint4 *>(S.m + pcs[0]);
    uint4 S0 = *reinterpret_cast<const uint4 *>(S.s + pcs[0]);
    uint4 L0 = make_uint4(0, 0, 0, 0), H0 = make_uint4(0, 0, 0, 0);  // starting sums (FR), in registers
    if (FR) {
        S0 = make_uint4(S0.x - 16, S0.y - 16, S0.z - 16, S0.w - 16);  // c = s - 16 of reduce_halves
        L0 = *reinterpret_cast<const uint4 *>(S.l0 + pcs[0]);
        H0 = *reinterpret_cast<const uint4 *>(S.h0 + pcs[0]);
    }
    uint32_t r0, r1;
    tma_group_rows(bk, g, &r0, &r1);
    const uint32_t gb = S.rp[r0], gn = S.rp[r1] - gb;
    const uint32_t RB = t.cw * 16u;
    uint4 *out = reinterpret_cast<uint4 *>(t.out) + (size_t)bk.row0 * t.C;
    const uint32_t C = t.C;
    const uint32_t gNS = g * bk.NS;
    Acc2 a[CPT][4];
    auto reset = [&]() {
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
            const bool own = k == 0 || same_primes;
            uint4 l = make_uint4(0, 0, 0, 0), h = l;  // zero sums unless FR
            if (FR) {
                l = own ? L0 : *reinterpret_cast<const uint4 *>(S.l0 + pcs[k]);
                h = own ? H0 : *reinterpret_cast<const uint4 *>(S.h0 + pcs[k]);
            }
            a[k][0] = Acc2{(int)l.x, (int)h.x};
            a[k][1] = Acc2{(int)l.y, (int)h.y};
            a[k][2] = Acc2{(int)l.z, (int)h.z};
            a[k][3] = Acc2{(int)l.w, (int)h.w};
        }
    };
    uint32_t r = r0;
    auto flush = [&]() {
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
            uint4 p = P0, m = M0, sh = S0;
            if (k > 0 && !same_primes) {
                p = *reinterpret_cast<const uint4 *>(S.p + pcs[k]);
                m = *reinterpret_cast<const uint4 *>(S.m + pcs[k]);
                sh = *reinterpret_cast<const uint4 *>(S.s + pcs[k]);
                if (FR) sh = make_uint4(sh.x - 16, sh.y - 16, sh.z - 16, sh.w - 16);
            }
            const uint4 v =
                FR ? make_uint4(reduce_halves(a[k][0], p.x, m.x, sh.x, FULL), reduce_halves(a[k][1], p.y, m.y, sh.y, FULL),
                                  reduce_halves(a[k][2], p.z, m.z, sh.z, FULL), reduce_halves(a[k][3], p.w, m.w, sh.w, FULL)) :
                FULL ? make_uint4(modred_reduce(acc_value(a[k][0], p.x), p.x, m.x, sh.x),
                                  modred_reduce(acc_value(a[k][1], p.y), p.y, m.y, sh.y),
                                  modred_reduce(acc_value(a[k][2], p.z), p.z, m.z, sh.z),
                                  modred_reduce(acc_value(a[k][3], p.w), p.w, m.w, sh.w))
                     : make_uint4(modred_reduce_signed(acc_value(a[k][0], p.x), p.x, m.x, sh.x),
                                  modred_reduce_signed(acc_value(a[k][1], p.y), p.y, m.y, sh.y),
                                  modred_reduce_signed(acc_value(a[k][2], p.z), p.z, m.z, sh.z),
                                  modred_reduce_signed(acc_value(a[k][3], p.w), p.w, m.w, sh.w));
            stcs128_if(out + (size_t)r * C + gcs[k], v, active[k]);
        }
        ++r;
        reset();
    };
    reset();
    // rows end where the next row's edges start; empty rows end at once
    while (r < r1 && S.rp[r + 1] == S.rp[r]) flush();
    uint32_t rend = r < r1 ? S.rp[r + 1] - gb : 0xffffffffu;  // group edge index one past row r's last
    uint32_t s = 0, ph = 0;
    for (uint32_t base = 0; base < gn; base += E) {
        const uint32_t st = gNS + s;
        if (!mbar_wait(smem_addr(&S.full_bar[st]), ph, S.deadline)) {
            atomicOr(err, 1);
            return;
        }
        int f[E];
        const uint32_t slot0 = st * E;
        if (E == 8) {
            const int4 c0 = *reinterpret_cast<const int4 *>(S.cf + slot0);
            const int4 c1 = *reinterpret_cast<const int4 *>(S.cf + slot0 + 4);
            f[0] = c0.x; f[1 % E] = c0.y; f[2 % E] = c0.z; f[3 % E] = c0.w;
            f[4 % E] = c1.x; f[5 % E] = c1.y; f[6 % E] = c1.z; f[7 % E] = c1.w;
        } else if (E == 4) {
            const int4 c0 = *reinterpret_cast<const int4 *>(S.cf + slot0);
            f[0] = c0.x; f[1 % E] = c0.y; f[2 % E] = c0.z; f[3 % E] = c0.w;
        } else if (E == 2) {
            const int2 c0 = *reinterpret_cast<const int2 *>(S.cf + slot0);
            f[0] = c0.x; f[1 % E] = c0.y;
        } else {
            f[0] = S.cf[slot0];
        }
        const uint32_t so = slot0 * RB;
#pragma unroll
        for (int j = 0; j < E; ++j) {
#pragma unroll
            for (int k = 0; k < CPT; ++k) {
                const uint32_t addr = col[k] + so + j * RB;
                const uint4 x = (PRED && k == 0) ? lds128_if(addr, deg0 >= S.sh[slot0 + j] ? 1u : 0u) : lds128(addr);
                mad_dp2a(a[k][0], x.x, f[j]);
                mad_dp2a(a[k][1], x.y, f[j]);
                mad_dp2a(a[k][2], x.z, f[j]);
                mad_dp2a(a[k][3], x.w, f[j]);
            }
            if (base + j + 1 == rend) {  // the last edge of row r (empty slots past gn never match)
                flush();
                while (r < r1 && S.rp[r + 1] == S.rp[r]) flush();
                rend = r < r1 ? S.rp[r + 1] - gb : 0xffffffffu;
            }
        }
        __syncwarp();
        mbar_arrive_if(smem_addr(&S.empty_bar[st]), lane == 0 ? 1u : 0u);
        if (++s == bk.NS) {
            s = 0;
            ph ^= 1u;
        }
    }
}

template <int E, int CPT, bool FR>
__device__ __forceinline__ void tma_dispatch(const GatherTask &t, const TmaBlock &bk, TmaShared &S, uint32_t ring_addr,
                                             uint32_t g, uint32_t c, uint32_t stride, int *err, bool pred) {
    if (t.partial) {
        if (pred) tma_consume<E, CPT, true, false, FR>(t, bk, S, ring_addr, g, c, stride, err);
        else tma_consume<E, CPT, false, false, FR>(t, bk, S, ring_addr, g, c, stride, err);
    } else {
        if (pred) tma_consume<E, CPT, true, true, FR>(t, bk, S, ring_addr, g, c, stride, err);
        else tma_consume<E, CPT, false, true, FR>(t, bk, S, ring_addr, g, c, stride, err);
    }
}

__host__ __device__ constexpr int tma_threads(int W) { return 32 * (1 + W); }

// W consumer warps: 8 / CPT (the wide block, 256 chunks per block) or
// kTmaNarrowWarps at CPT 1 (160 chunks, one row group).
template <int E, int CPT, int W>
__global__ void __launch_bounds__(tma_threads(W), tma_min_blocks(E, CPT, W == kTmaConsumers / CPT ? 0 : W))
    gather_tma_kernel(const GatherTask *__restrict__ tasks, int n_tasks, uint32_t rpb, uint32_t ring_bytes, int *err) {
    extern __shared__ __align__(128) uint8_t ring[];
    __shared__ TmaShared S;
    constexpr uint32_t kCover = 32u * W * CPT;  // chunks one block covers

    if (threadIdx.x == 0) S.abort_flag = *(volatile int *)err;  // a previous block gave up: do nothing
    __syncthreads();
    if (S.abort_flag) return;
    int lo = 0, hi = n_tasks - 1;
    const uint32_t b = blockIdx.x;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (tasks[mid].block_begin <= b) lo = mid; else hi = mid - 1;
    }
    if (threadIdx.x == 0) S.task = tasks[lo];
    __syncthreads();
    const GatherTask &t = S.task;
    TmaBlock bk;
    uint32_t rb = b - t.block_begin;  // row block of this block
    if (t.block_order) rb = __ldg(t.block_order + block_order_offset(t.rows, rpb) + rb);
    bk.row0 = rb * rpb;
    bk.nrows = min(rpb, t.rows - bk.row0);
    const uint32_t RB = t.cw * 16u;
    bk.G = 1;  // row groups: each group's warps cover kCover / G chunks (G divides W)
    while (W % (2 * bk.G) == 0 && 2 * bk.G * t.cw <= kCover) bk.G *= 2;
    const uint32_t slots_g = min((uint32_t)kTmaMaxSlots / bk.G, ring_bytes / (bk.G * RB));
    bk.NS = slots_g / E;                                 // stages per group
    const uint32_t wpg = W / bk.G;                       // consumer warps per group
    bk.act = min(wpg, (t.cw + 31) / 32);                 // warps with chunks, per group
    if (bk.NS == 0 || bk.G * E > 32 || t.cw > kCover || t.cw == 0 || rpb > (uint32_t)kTmaMaxRows) {  // refusal
        if (threadIdx.x == 0) atomicOr(err, 8);
        return;
    }
    for (uint32_t i = threadIdx.x; i <= bk.nrows; i += blockDim.x) S.rp[i] = __ldg(t.row_ptr + bk.row0 + i);
    if (threadIdx.x < t.n_primes) {
        const ModRed mr = modred_make(__ldg(t.primes + threadIdx.x));
        S.p[threadIdx.x] = mr.p;
        S.m[threadIdx.x] = mr.m;
        S.s[threadIdx.x] = mr.s;
        S.l0[threadIdx.x] = (mr.p & 1u) << 15;
        S.h0[threadIdx.x] = mr.p >> 1;
    }
    if (threadIdx.x == 0) {
        for (uint32_t s = 0; s < bk.G * bk.NS; ++s) {
            mbar_init(smem_addr(&S.full_bar[s]), E);
            mbar_init(smem_addr(&S.empty_bar[s]), bk.act);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        S.deadline = clock64() + kWaitCycles;
    }
    // every prime at least 2^17: the consumers start the sums at p 2^15 and reduce in
    // 32-bit arithmetic (reduce_halves); otherwise from zero, in 64 bits (the two paths are
    // separate instantiations: one kernel body holding both ran slower)
    const bool fr =
        __syncthreads_and(threadIdx.x >= t.n_primes || S.p[threadIdx.x] >= (1u << 17)) != 0;
    const uint32_t warp = threadIdx.x >> 5;
    if (warp == 0) {
        tma_produce<E>(t, bk, S, ring, err);
        return;
    }
    const uint32_t cwi = warp - 1;
    const uint32_t g = cwi / wpg, wi = cwi - g * wpg;
    if (wi >= bk.act) return;  // all of this warp's chunks lie beyond the row
    const uint32_t c = wi * 32 + (threadIdx.x & 31);
    const uint32_t stride = 32 * wpg;  // chunks the group's warps cover side by side
    const uint32_t ring_addr = smem_addr(ring);
    const bool pred = t.c0 + wi * 32 < (uint32_t)kTmaMaxShift * t.cpd;
    if (fr)
        tma_dispatch<E, CPT, true>(t, bk, S, ring_addr, g, c, stride, err, pred);
    else
        tma_dispatch<E, CPT, false>(t, bk, S, ring_addr, g, c, stride, err, pred);
}

// Ring sizes: ring_kb KB per block (several blocks per SM).
constexpr uint32_t kTmaRingMax = 192 * 1024;
constexpr uint32_t kTmaRingMin = 16 * 1024;

bool tma_usable(const GatherTask &t) { return t.vec4 && t.cw >= 1 && t.cw <= 256 && t.small_coefs; }

template <int E, int CPT, int W>
static int set_attr() {
    CP_CUDA_TRY(cudaFuncSetAttribute(gather_tma_kernel<E, CPT, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kTmaRingMax));
    return CP_OK;
}

template <int CPT, int W>
static int set_attrs() {
    int rc;
    if ((rc = set_attr<1, CPT, W>()) || (rc = set_attr<2, CPT, W>()) || (rc = set_attr<4, CPT, W>()) ||
        (rc = set_attr<8, CPT, W>()))
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
    if ((rc = set_attrs<1, kTmaConsumers>()) || (rc = set_attrs<2, kTmaConsumers / 2>()) ||
        (rc = set_attrs<4, kTmaConsumers / 4>()) || (rc = set_attrs<1, kTmaNarrowWarps>()))
        return rc;
    done[dev] = true;
    return CP_OK;
}

template <int CPT, int W>
static int launch_cpt(const GatherTask *tasks_dev, int n_tasks, uint32_t blocks, uint32_t rpb, uint32_t dyn, int *err,
                      cudaStream_t st, int edges) {
    constexpr int T = tma_threads(W);
    switch (edges) {
        case 1: gather_tma_kernel<1, CPT, W><<<blocks, T, dyn, st>>>(tasks_dev, n_tasks, rpb, dyn, err); break;
        case 2: gather_tma_kernel<2, CPT, W><<<blocks, T, dyn, st>>>(tasks_dev, n_tasks, rpb, dyn, err); break;
        case 4: gather_tma_kernel<4, CPT, W><<<blocks, T, dyn, st>>>(tasks_dev, n_tasks, rpb, dyn, err); break;
        case 8: gather_tma_kernel<8, CPT, W><<<blocks, T, dyn, st>>>(tasks_dev, n_tasks, rpb, dyn, err); break;
        default: return fail(CP_EINVAL, "TMA gather edges per stage must be 1, 2, 4 or 8");
    }
    return CP_OK;
}

// rpb: destination rows per block (16..128); edges: edges per stage (1, 2, 4 or 8);
// cpt: 16-byte chunks per consumer thread (1, 2 or 4); ring_kb: shared-memory ring per block;
// narrow: 5 consumer warps (cpt 1, rows of at most 160 chunks) instead of 8 / cpt.
int launch_gather_tma(const GatherTask *tasks_dev, int n_tasks, uint32_t total_blocks, int rpb, int *err,
                      cudaStream_t st, int edges, int ring_kb, int cpt, bool narrow) {
    if (n_tasks <= 0 || total_blocks == 0) return CP_OK;
    if (rpb != 16 && rpb != 32 && rpb != 64 && rpb != 128)
        return fail(CP_EINVAL, "TMA gather rows per block must be 16, 32, 64 or 128");
    uint32_t dyn = (uint32_t)ring_kb * 1024u;
    if (dyn < kTmaRingMin) dyn = kTmaRingMin;
    if (dyn > kTmaRingMax) dyn = kTmaRingMax;
    int rc;
    if (narrow && cpt != 1) return fail(CP_EINVAL, "narrow TMA gather blocks take one chunk per thread");
    switch (cpt) {
        case 1:
            rc = narrow ? launch_cpt<1, kTmaNarrowWarps>(tasks_dev, n_tasks, total_blocks, rpb, dyn, err, st, edges)
                        : launch_cpt<1, kTmaConsumers>(tasks_dev, n_tasks, total_blocks, rpb, dyn, err, st, edges);
            break;
        case 2: rc = launch_cpt<2, kTmaConsumers / 2>(tasks_dev, n_tasks, total_blocks, rpb, dyn, err, st, edges); break;
        case 4: rc = launch_cpt<4, kTmaConsumers / 4>(tasks_dev, n_tasks, total_blocks, rpb, dyn, err, st, edges); break;
        default: return fail(CP_EINVAL, "TMA gather chunks per thread must be 1, 2 or 4");
    }
    if (rc) return rc;
    CP_CUDA_TRY(cudaGetLastError());
    return CP_OK;
}

}  // namespace cp

// Diagnostic: reduce_halves on given word sums (one thread per value).
namespace cp {
__global__ void debug_halves_kernel(const int *lo, const int *hi, const uint32_t *pr, int n, int full, uint32_t *out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const ModRed mr = modred_make(pr[k]);
    out[k] = reduce_halves(Acc2{lo[k], hi[k]}, mr.p, mr.m, mr.s - 16, full != 0);
}
}  // namespace cp

extern "C" int cp_debug_reduce_halves(const int32_t *lo_host, const int32_t *hi_host, const uint32_t *p_host, int n,
                                      int full, uint32_t *out_host) {
    using namespace cp;
    if (n < 0 || (n > 0 && (!lo_host || !hi_host || !p_host || !out_host))) return fail(CP_EINVAL, "bad arguments");
    for (int k = 0; k < n; ++k) {
        const uint32_t p = p_host[k];
        if (p < (1u << 17) || p >= (1u << 31)) return fail(CP_EINVAL, "p must be in [2^17, 2^31)");
        const long long u = (long long)hi_host[k] * 65536 + lo_host[k];
        if (u <= 0 || u >= (long long)p * 65536) return fail(CP_EINVAL, "hi 2^16 + lo must lie in (0, p 2^16)");
    }
    if (n == 0) return CP_OK;
    int *lo_d = nullptr, *hi_d = nullptr;
    uint32_t *p_d = nullptr, *o_d = nullptr;
    int rc = dev_alloc((void **)&lo_d, 4ull * n);
    if (!rc) rc = dev_alloc((void **)&hi_d, 4ull * n);
    if (!rc) rc = dev_alloc((void **)&p_d, 4ull * n);
    if (!rc) rc = dev_alloc((void **)&o_d, 4ull * n);
    cudaError_t e = cudaSuccess;
    if (!rc) {
        e = cudaMemcpy(lo_d, lo_host, 4ull * n, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(hi_d, hi_host, 4ull * n, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(p_d, p_host, 4ull * n, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) {
            debug_halves_kernel<<<(n + 255) / 256, 256>>>(lo_d, hi_d, p_d, n, full, o_d);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpy(out_host, o_d, 4ull * n, cudaMemcpyDeviceToHost);
    }
    dev_free(lo_d);
    dev_free(hi_d);
    dev_free(p_d);
    dev_free(o_d);
    if (rc) return rc;
    if (e != cudaSuccess) return fail(CP_ECUDA, std::string("cp_debug_reduce_halves: ") + cudaGetErrorString(e));
    return CP_OK;
}
