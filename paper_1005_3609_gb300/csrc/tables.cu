// Transition tables of the per-site factors, built on the GPU.
//
// For every source state of a factor's input space: unrank it, apply the
// factor's single-edge operators (Sec. 3.1-3.3), drop the terms the
// projectors kill, rank each surviving partition in the output space, and
// emit (dst, src, shift, coef) terms.  The terms are then counting-sorted by
// destination into a CSR table, so that the per-site kernel is a gather.
// Tables depend only on (lattice, L, site): they are built once per device
// and shared by every strip, row, height and prime.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <utility>

#include "cp_internal.h"
#include "modred.cuh"
#include "ncnnn.cuh"

namespace cp {

// ------------------------------------------------------------------ rank tables

// cnt and off from the recursion M_p = M_{p-1} + sum_{k=0}^{p-2} M_k M_{p-k-2}, eq. (M_recurs).
__global__ void rank_tables_kernel(RankTables *T) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    uint64_t M[kTblStride];
    M[0] = 1;
    M[1] = 1;
    for (int p = 2; p < kTblStride; ++p) {
        uint64_t s = M[p - 1];
        for (int k = 0; k <= p - 2; ++k) s += M[k] * M[p - k - 2];
        M[p] = s;
    }
    T->cnt[0] = 1;
    for (int n = 1; n < kTblStride; ++n) T->cnt[n] = M[n - 1];
    for (int k = 0; k < kTblStride * kTblStride; ++k) T->off[k] = 0;
    for (int n = 3; n < kTblStride; ++n) {
        uint64_t o = T->cnt[n - 1];
        for (int k = 0; k <= n - 3; ++k) {
            T->off[n * kTblStride + k] = o;
            o += T->cnt[k + 1] * T->cnt[n - k - 2];
        }
    }
    // Catalan numbers and the offsets of the non-crossing order (partner at 1+k)
    T->cntc[0] = 1;
    for (int n = 1; n < kTblStride; ++n) {
        uint64_t c = 0;
        for (int k = 0; k < n; ++k) c += T->cntc[k] * T->cntc[n - 1 - k];
        T->cntc[n] = c;
    }
    for (int k = 0; k < kTblStride * kTblStride; ++k) T->offc[k] = 0;
    for (int n = 2; n < kTblStride; ++n) {
        uint64_t o = T->cntc[n - 1];
        for (int k = 0; k <= n - 2; ++k) {
            T->offc[n * kTblStride + k] = o;
            o += T->cntc[k] * T->cntc[n - 1 - k];
        }
    }
}

// ------------------------------------------------------------------ term generation

struct Term {
    Labels s;
    int32_t coef;
    int32_t shift;
};

constexpr int kMaxTerms = 8;   // terms of one factor applied to one partition
constexpr int kMaxFused = 64;  // terms of a two-site table before merging

// H_{a,b} = 1 - J_{a,b} at v = -1: a term with a ~ b is killed (H s = s - s), otherwise
// it splits into itself and the joined partition with -w.
__device__ int op_h(Term *t, int n, int m, int a, int b) {
    int k = n;
    for (int j = 0; j < n; ++j) {
        if (t[j].s.v[a] == t[j].s.v[b]) { t[j].coef = 0; continue; }
        Term u = t[j];
        join_blocks(u.s, m, a, b);
        u.coef = -u.coef;
        u.shift += 1;
        t[k++] = u;
    }
    int w = 0;
    for (int j = 0; j < k; ++j)
        if (t[j].coef != 0) t[w++] = t[j];
    return w;
}

// V_i = D_i - w.
__device__ int op_v(Term *t, int n, int m, int i) {
    for (int j = 0; j < n; ++j) {
        Term u = t[j];
        u.coef = -u.coef;
        u.shift += 1;
        t[n + j] = u;
        detach_site(t[j].s, m, i);
    }
    return 2 * n;
}

__device__ int op_d(Term *t, int n, int m, int i) {
    for (int j = 0; j < n; ++j) detach_site(t[j].s, m, i);
    return n;
}

// P_{j,j+1} for j in [lo, hi) except `skip`.
__device__ int op_p(Term *t, int n, int lo, int hi, int skip) {
    int w = 0;
    for (int j = 0; j < n; ++j) {
        bool ok = true;
        for (int q = lo; q < hi; ++q)
            if (q != skip && t[j].s.v[q] == t[j].s.v[q + 1]) { ok = false; break; }
        if (ok) t[w++] = t[j];
    }
    return w;
}

// Any-v operators (Sec. 3.1): H_{a,b} = 1 + v J_{a,b}, where J is the identity
// (no w) when a ~ b and joins with a factor w otherwise; V_i = v w + D_i.
__device__ int op_hv(Term *t, int n, int m, int a, int b, int v) {
    int k = n;
    for (int j = 0; j < n; ++j) {
        if (t[j].s.v[a] == t[j].s.v[b]) {
            t[j].coef *= (1 + v);
            continue;
        }
        Term u = t[j];
        join_blocks(u.s, m, a, b);
        u.coef *= v;
        u.shift += 1;
        t[k++] = u;
    }
    int w = 0;
    for (int j = 0; j < k; ++j)
        if (t[j].coef != 0) t[w++] = t[j];
    return w;
}

__device__ int op_vv(Term *t, int n, int m, int i, int v) {
    for (int j = 0; j < n; ++j) {
        Term u = t[j];
        u.coef *= v;
        u.shift += 1;
        t[n + j] = u;
        detach_site(t[j].s, m, i);
    }
    int w = 0;
    for (int j = 0; j < 2 * n; ++j)
        if (t[j].coef != 0) t[w++] = t[j];
    return w;
}

// Terms of one factor applied to one partition.
__device__ __noinline__ int factor_terms(const OpDesc &op, const Labels &s, Term *t) {
    int m = op.m, i = op.i, n = 1;
    t[0].s = s;
    t[0].coef = 1;
    t[0].shift = 0;
    switch (op.kind) {
        case OP_SQUARE:  // (prod_{j!=i} P) V_i H_{i,i+1};  T_m = (prod P) V_m      eq. (T_sq_proj)
            if (i < m - 1) n = op_h(t, n, m, i, i + 1);
            n = op_v(t, n, m, i);
            n = op_p(t, n, 0, m - 1, i < m - 1 ? i : -1);
            break;
        case OP_TRIANGULAR:  // (prod P) V_i H_{i-1,i} H_{i,i+1}                    Sec. 3.3
            if (i < m - 1) n = op_h(t, n, m, i, i + 1);
            if (i > 0) n = op_h(t, n, m, i - 1, i);
            n = op_v(t, n, m, i);
            n = op_p(t, n, 0, m - 1, -1);
            break;
        case OP_LAST:  // (prod_{j>i} P) D_i H_{i,i+1}                                eq. (T_last_i)
            if (i < m - 1) n = op_h(t, n, m, i, i + 1);
            n = op_d(t, n, m, i);
            n = op_p(t, n, i + 1, m - 1, -1);
            break;
        case OP_POTTS_SQUARE:  // V_i H_{i,i+1}: the rows of T = (prod V)(prod H), Sec. 3.2
            if (i < m - 1) n = op_hv(t, n, m, i, i + 1, op.v);
            n = op_vv(t, n, m, i, op.v);
            break;
        case OP_POTTS_TRIANGULAR:  // V_i H_{i-1,i} H_{i,i+1} (H_{i-1,i}: the diagonal, Sec. 3.3)
            if (i < m - 1) n = op_hv(t, n, m, i, i + 1, op.v);
            if (i > 0) n = op_hv(t, n, m, i - 1, i, op.v);
            n = op_vv(t, n, m, i, op.v);
            break;
        case OP_POTTS_LAST:  // D_i H_{i,i+1}: last horizontal edges; every state ends at e_0
            if (i < m - 1) n = op_hv(t, n, m, i, i + 1, op.v);
            n = op_d(t, n, m, i);
            break;
        default:  // identity
            break;
    }
    return n;
}

// Terms of a two-site table: the second factor applied to every term of the first.
__device__ __noinline__ int fused_terms(const OpDesc &op, const Labels &s, Term *out) {
    Term a[kMaxTerms];
    const int na = factor_terms(op, s, a);
    OpDesc ob = op;
    ob.kind = op.kind_b;
    ob.i = op.i_b;
    int n = 0;
    for (int j = 0; j < na; ++j) {
        Term b[kMaxTerms];
        const int nb = factor_terms(ob, a[j].s, b);
        for (int q = 0; q < nb; ++q) {
            out[n].s = b[q].s;
            out[n].coef = a[j].coef * b[q].coef;
            out[n].shift = a[j].shift + b[q].shift;
            ++n;
        }
    }
    return n;
}

// One thread per source state.  slot_dst[src*K + t] = destination rank or ~0u,
// slot_edge[...] = packed edge.  err bits: 1 bad rank / membership, 2 too many
// terms, 4 coefficient out of range, 8 unrank/rank mismatch of the source.
template <int NT>
__global__ void build_terms_kernel(OpDesc op, const RankTables *Tg, uint32_t *slot_dst, uint32_t *slot_edge,
                                   int K, int *err) {
    __shared__ RankTables T;
    stage_tables(T, Tg);
    uint64_t src = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (src >= op.in.size) return;
    Labels s;
    space_unrank(src, op.in, s, T);
    int bad = 0;
    if (!space_contains(s, op.in) || space_rank(s, op.in, T) != src) bad |= 8;
    Term t[NT];
    int n = op.fused ? fused_terms(op, s, t) : factor_terms(op, s, t);
    uint32_t dst[NT];
    for (int j = 0; j < n; ++j) {
        if (!space_contains(t[j].s, op.out)) { bad |= 1; dst[j] = ~0u; continue; }
        uint64_t r = space_rank(t[j].s, op.out, T);
        if (r >= op.out.size) { bad |= 1; dst[j] = ~0u; continue; }
        dst[j] = (uint32_t)r;
    }
    // merge equal (dst, shift)
    for (int j = 0; j < n; ++j) {
        if (t[j].coef == 0 || dst[j] == ~0u) continue;
        for (int q = j + 1; q < n; ++q)
            if (dst[q] == dst[j] && t[q].shift == t[j].shift && t[q].coef != 0) {
                t[j].coef += t[q].coef;
                t[q].coef = 0;
            }
    }
    const int sb = op.src_bits, cb = 30 - sb;  // coefficient bits
    const int cmin = -(1 << (cb - 1)), cmax = (1 << (cb - 1)) - 1;
    int w = 0;
    for (int j = 0; j < n; ++j) {
        if (t[j].coef == 0 || dst[j] == ~0u) continue;
        if (t[j].coef < cmin || t[j].coef > cmax || t[j].shift > 3) { bad |= 4; continue; }
        if (w >= K) { bad |= 2; break; }
        slot_dst[src * K + w] = dst[j];
        slot_edge[src * K + w] = (uint32_t)src | ((uint32_t)t[j].shift << sb) |
                                 (((uint32_t)t[j].coef & ((1u << cb) - 1u)) << (sb + 2));
        ++w;
    }
    for (; w < K; ++w) slot_dst[src * K + w] = ~0u;
    if (bad) atomicOr(err, bad);
}

// ------------------------------------------------------------------ CSR by destination

// Edges per destination, and sum of |coef| per destination into csum.
__global__ void count_kernel(const uint32_t *slot_dst, const uint32_t *slot_edge, uint64_t n_slots, int src_bits,
                             uint32_t *cnt, uint32_t *csum, int *max_coef) {
    uint32_t m = 0;  // largest |coefficient| seen by this thread
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_slots;
         k += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t d = slot_dst[k];
        if (d == ~0u) continue;
        atomicAdd(&cnt[d], 1u);
        const int c = (int)slot_edge[k] >> (src_bits + 2);
        const uint32_t a = (uint32_t)(c < 0 ? -c : c);
        atomicAdd(&csum[d], a);
        m = max(m, a);
    }
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(max_coef, (int)m);
}

// Largest entry of cnt (warp maximum, one atomic per warp).
__global__ void max_count_kernel(const uint32_t *cnt, uint64_t n, int *out) {
    uint32_t m = 0;
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (uint64_t)gridDim.x * blockDim.x)
        m = max(m, cnt[k]);
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (int)m);
}

constexpr int kScanThreads = 1024;

// Exclusive scan, three passes: per-block sums, scan of the block sums, per-block scan + offset.
__device__ __forceinline__ uint32_t block_inclusive_scan(uint32_t v, uint32_t *warp_sums) {
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) warp_sums[wid] = v;
    __syncthreads();
    if (wid == 0) {
        uint32_t x = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        warp_sums[lane] = x;
    }
    __syncthreads();
    if (wid > 0) v += warp_sums[wid - 1];
    return v;
}

__global__ void scan_block_sums(const uint32_t *in, uint64_t n, uint32_t *block_sums) {
    __shared__ uint32_t ws[32];
    uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t v = k < n ? in[k] : 0;
    uint32_t s = block_inclusive_scan(v, ws);
    if (threadIdx.x == blockDim.x - 1) block_sums[blockIdx.x] = s;
}

__global__ void scan_sums_serial(uint32_t *sums, uint32_t n_blocks) {
    // single block: exclusive scan of the block sums in chunks of blockDim
    __shared__ uint32_t ws[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < n_blocks; base += blockDim.x) {
        uint32_t k = base + threadIdx.x;
        uint32_t v = k < n_blocks ? sums[k] : 0;
        uint32_t inc = block_inclusive_scan(v, ws);
        uint32_t c = carry;
        if (k < n_blocks) sums[k] = c + inc - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = c + inc;
        __syncthreads();
    }
}

__global__ void scan_finish(const uint32_t *in, uint64_t n, const uint32_t *block_off, uint32_t *out) {
    __shared__ uint32_t ws[32];
    uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t v = k < n ? in[k] : 0;
    uint32_t inc = block_inclusive_scan(v, ws);
    uint32_t exc = block_off[blockIdx.x] + inc - v;
    if (k < n) out[k] = exc;
    if (k == n - 1) out[n] = exc + v;
}

__global__ void fill_kernel(const uint32_t *slot_dst, const uint32_t *slot_edge, uint64_t n_slots,
                            const uint32_t *row_ptr, uint32_t *cursor, uint32_t *edges) {
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_slots;
         k += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t d = slot_dst[k];
        if (d == ~0u) continue;
        uint32_t pos = row_ptr[d] + atomicAdd(&cursor[d], 1u);
        edges[pos] = slot_edge[k];
    }
}

// Deterministic order inside each destination: by packed value (src, then shift/coef).
__global__ void sort_segments_kernel(const uint32_t *row_ptr, uint64_t n_dst, uint32_t *edges) {
    uint64_t d = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= n_dst) return;
    uint32_t b = row_ptr[d], e = row_ptr[d + 1];
    for (uint32_t i = b + 1; i < e; ++i) {
        uint32_t x = edges[i];
        uint32_t j = i;
        while (j > b && edges[j - 1] > x) {
            edges[j] = edges[j - 1];
            --j;
        }
        edges[j] = x;
    }
}

// flag[b] = 1 if the NCNNN partition of rank b has e alone and e-1 !~ e+1, so that
// J_{e,e+1} of it lies in X_e (every partition of X_e with e ~ e+1 arises once).
__global__ void x_partner_kernel(int m, int e, const RankTables *Tg, uint32_t *flag) {
    __shared__ RankTables T;
    stage_tables(T, Tg);
    uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= T.cnt[m]) return;
    Labels s;
    ncnnn_unrank(b, 0, m, s, T);
    bool alone = true;
    for (int i = 0; i < m; ++i)
        if (i != e && s.v[i] == s.v[e]) alone = false;
    flag[b] = (alone && (e == 0 || s.v[e - 1] != s.v[e + 1])) ? 1u : 0u;
}

// ------------------------------------------------------------------ host side

static int scan_exclusive(const uint32_t *cnt, uint64_t n, uint32_t *row_ptr, cudaStream_t st) {
    uint64_t nb = (n + kScanThreads - 1) / kScanThreads;
    if (nb > (1u << 31)) return fail(CP_EINVAL, "scan too large");
    uint32_t *sums = nullptr;
    int rc = dev_alloc((void **)&sums, (nb + 1) * sizeof(uint32_t));
    if (rc) return rc;
    scan_block_sums<<<(unsigned)nb, kScanThreads, 0, st>>>(cnt, n, sums);
    scan_sums_serial<<<1, kScanThreads, 0, st>>>(sums, (uint32_t)nb);
    scan_finish<<<(unsigned)nb, kScanThreads, 0, st>>>(cnt, n, sums, row_ptr);
    cudaError_t e = cudaGetLastError();
    cudaStreamSynchronize(st);
    dev_free(sums);
    if (e != cudaSuccess) return fail(CP_ECUDA, std::string("scan: ") + cudaGetErrorString(e));
    return CP_OK;
}

int build_x_prefix(int m, int e, cudaStream_t st, uint32_t **out) {
    const RankTables *T_dev = nullptr;
    RankTables T;
    int rc = device_rank_tables(&T_dev, &T);
    if (rc) return rc;
    const uint64_t Sb = T.cnt[m];
    uint32_t *flag = nullptr, *pre = nullptr;
    if ((rc = dev_alloc((void **)&flag, Sb * 4))) return rc;
    if ((rc = dev_alloc((void **)&pre, (Sb + 1) * 4))) {
        dev_free(flag);
        return rc;
    }
    x_partner_kernel<<<(unsigned)((Sb + 127) / 128), 128, 0, st>>>(m, e, T_dev, flag);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) {
        dev_free(flag);
        dev_free(pre);
        return fail(CP_ECUDA, std::string("x_partner: ") + cudaGetErrorString(ce));
    }
    rc = scan_exclusive(flag, Sb, pre, st);
    dev_free(flag);
    if (rc) {
        dev_free(pre);
        return rc;
    }
    uint32_t total = 0;
    CP_CUDA_TRY(cudaMemcpy(&total, pre + Sb, 4, cudaMemcpyDeviceToHost));
    if (total != T.cnt[m - 1]) {
        dev_free(pre);
        return fail(CP_ESTATE, "excepted space has the wrong size");
    }
    *out = pre;
    return CP_OK;
}

// Smallest source state of each row block of `rpb` destination rows (one warp
// per block; a block without edges gets 0xffffffff).
__global__ void block_min_src_kernel(const uint32_t *row_ptr, const uint32_t *edges, uint32_t n_dst, uint32_t mask,
                                     uint32_t rpb, uint32_t nb, uint32_t *key) {
    const uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= nb) return;
    const uint32_t r0 = w * rpb, r1 = min(n_dst, r0 + rpb);
    const uint32_t e1 = row_ptr[r1];
    uint32_t m = 0xffffffffu;
    for (uint32_t e = row_ptr[r0] + lane; e < e1; e += 32) m = min(m, edges[e] & mask);
    m = __reduce_min_sync(0xffffffffu, m);
    if (lane == 0) key[w] = m;
}

constexpr uint64_t kBlockOrderMinRows = 4096;  // smaller tables keep row-block order

// The order in which the TMA gather's blocks visit a table's row blocks: by
// the smallest source state a row block reads (ties in row order), for each
// rows-per-block choice.  Destinations whose sources lie close together then
// run at the same time, so a source row fetched into L2 serves the blocks that
// need it before it is evicted -- the factors of the first sites of a row draw
// their sources from the whole state vector in rank order.  Any order gives
// the same results; this one only changes DRAM traffic.
static int build_block_order(SiteTable *tab, cudaStream_t st) {
    if (tab->n_dst < kBlockOrderMinRows || tab->nnz == 0) return CP_OK;
    const uint32_t n = (uint32_t)tab->n_dst;
    const uint32_t total = block_order_offset(n, 256);  // 16, 32, 64 and 128 rows per block
    uint32_t *key = nullptr;
    int rc = dev_alloc((void **)&key, (size_t)total * 4);
    if (rc) return rc;
    const uint32_t mask = (1u << tab->op.src_bits) - 1u;
    for (uint32_t l = 16; l <= 128; l *= 2) {
        const uint32_t nb = (n + l - 1) / l;
        block_min_src_kernel<<<(nb + 7) / 8, 256, 0, st>>>(tab->row_ptr, tab->edges, n, mask, l, nb,
                                                           key + block_order_offset(n, l));
    }
    std::vector<uint32_t> hk(total), order(total);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(hk.data(), key, (size_t)total * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dev_free(key);
    if (e != cudaSuccess) return fail(CP_ECUDA, std::string("block order: ") + cudaGetErrorString(e));
    for (uint32_t l = 16; l <= 128; l *= 2) {
        const uint32_t off = block_order_offset(n, l), nb = (n + l - 1) / l;
        uint32_t *o = order.data() + off;
        for (uint32_t i = 0; i < nb; ++i) o[i] = i;
        std::stable_sort(o, o + nb, [&](uint32_t a, uint32_t b) { return hk[off + a] < hk[off + b]; });
    }
    if ((rc = dev_alloc((void **)&tab->block_order, (size_t)total * 4))) return rc;
    CP_CUDA_TRY(cudaMemcpy(tab->block_order, order.data(), (size_t)total * 4, cudaMemcpyHostToDevice));
    return CP_OK;
}

static int build_table(const OpDesc &op, const RankTables *T_dev, cudaStream_t st, SiteTable *tab) {
    tab->op = op;
    tab->n_src = op.in.size;
    tab->n_dst = op.out.size;
    tab->n_site_out = op.out.size;
    if (op.in.size > ((1ull << op.src_bits) - 1) || op.out.size >= 0xFFFFFFFFull)
        return fail(CP_EINVAL, "state space too large for the edge format");
    const int K = op.max_terms;
    uint64_t n_slots = op.in.size * (uint64_t)K;
    uint32_t *slot_dst = nullptr, *slot_edge = nullptr, *cnt = nullptr, *cursor = nullptr, *csum = nullptr;
    int *err = nullptr;
    int rc = CP_OK;
    auto cleanup = [&]() {
        dev_free(slot_dst);
        dev_free(slot_edge);
        dev_free(cnt);
        dev_free(cursor);
        dev_free(csum);
        dev_free(err);
    };
    if ((rc = dev_alloc((void **)&slot_dst, n_slots * 4)) || (rc = dev_alloc((void **)&slot_edge, n_slots * 4)) ||
        (rc = dev_alloc((void **)&cnt, op.out.size * 4)) || (rc = dev_alloc((void **)&cursor, op.out.size * 4)) ||
        (rc = dev_alloc((void **)&csum, op.out.size * 4)) ||
        (rc = dev_alloc((void **)&err, 3 * sizeof(int)))) {
        cleanup();
        return rc;
    }
    if ((rc = dev_alloc((void **)&tab->row_ptr, (op.out.size + 1) * 4))) {
        cleanup();
        return rc;
    }
    cudaMemsetAsync(cnt, 0, op.out.size * 4, st);
    cudaMemsetAsync(cursor, 0, op.out.size * 4, st);
    cudaMemsetAsync(csum, 0, op.out.size * 4, st);
    cudaMemsetAsync(err, 0, 3 * sizeof(int), st);
    const int bt = 128;
    if (op.fused)
        build_terms_kernel<kMaxFused><<<(unsigned)((op.in.size + bt - 1) / bt), bt, 0, st>>>(op, T_dev, slot_dst,
                                                                                            slot_edge, K, err);
    else
        build_terms_kernel<kMaxTerms><<<(unsigned)((op.in.size + bt - 1) / bt), bt, 0, st>>>(op, T_dev, slot_dst,
                                                                                            slot_edge, K, err);
    count_kernel<<<1216, 256, 0, st>>>(slot_dst, slot_edge, n_slots, op.src_bits, cnt, csum, err + 2);
    max_count_kernel<<<608, 256, 0, st>>>(csum, op.out.size, err + 1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        cleanup();
        return fail(CP_ECUDA, std::string("build_terms: ") + cudaGetErrorString(e));
    }
    if ((rc = scan_exclusive(cnt, op.out.size, tab->row_ptr, st))) {
        cleanup();
        return rc;
    }
    int herr[3] = {0, 0, 0};
    uint32_t nnz = 0;
    cudaMemcpyAsync(herr, err, 3 * sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&nnz, tab->row_ptr + op.out.size, 4, cudaMemcpyDeviceToHost, st);
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cleanup();
        return fail(CP_ECUDA, std::string("table build: ") + cudaGetErrorString(e));
    }
    // The gathers reduce p 2^21 + sum_e coef_e x_e (x_e < p) exactly while
    // sum_e |coef_e| into every state stays below 2^20 (modred.cuh).
    if (herr[0] == 0 && herr[1] >= (int)kReduceMaxCoefSum) {
        cleanup();
        return fail(CP_EINVAL, "too many transitions into one state for the exact modular reduction");
    }
    if (herr[0] == 4) {
        cleanup();
        return fail(CP_EINVAL, "a transition coefficient does not fit the " + std::to_string(30 - op.src_bits) +
                                   "-bit field of this width's edge format (|v| too large)");
    }
    if (herr[0]) {
        cleanup();
        return fail(CP_ESTATE, "transition table check failed (flags " + std::to_string(herr[0]) + ") for op kind " +
                                   std::to_string(op.kind) + " m=" + std::to_string(op.m) + " i=" +
                                   std::to_string(op.i));
    }
    tab->nnz = nnz;
    tab->max_coef_sum = (uint32_t)herr[1];
    tab->max_abs_coef = (uint32_t)herr[2];
    if ((rc = dev_alloc((void **)&tab->edges, (size_t)(nnz ? nnz : 1) * 4))) {
        cleanup();
        return rc;
    }
    fill_kernel<<<1216, 256, 0, st>>>(slot_dst, slot_edge, n_slots, tab->row_ptr, cursor, tab->edges);
    sort_segments_kernel<<<(unsigned)((op.out.size + 255) / 256), 256, 0, st>>>(tab->row_ptr, op.out.size, tab->edges);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cleanup();
    if (e != cudaSuccess) return fail(CP_ECUDA, std::string("csr fill: ") + cudaGetErrorString(e));
    return build_block_order(tab, st);
}

TableSet::~TableSet() {
    for (auto p : x_prefix) dev_free(p);
    for (auto &t : row) {
        dev_free(t.row_ptr);
        dev_free(t.edges);
        dev_free(t.block_order);
    }
    for (auto &t : last) {
        dev_free(t.row_ptr);
        dev_free(t.edges);
        dev_free(t.block_order);
    }
}

// Identity factor on a 1-state space (T_1^last = D_1 on the width-1 strip).
static int identity_table(int m, SiteTable *tab) {
    OpDesc op{};
    op.kind = OP_IDENTITY;
    op.m = m;
    op.src_bits = (int)kSrcBits;
    op.in = Space{SPACE_B, m, 0, 0, 1, nullptr};
    op.out = op.in;
    tab->op = op;
    tab->n_src = tab->n_dst = tab->nnz = tab->n_site_out = 1;
    tab->max_coef_sum = tab->max_abs_coef = 1;
    int rc = dev_alloc((void **)&tab->row_ptr, 8);
    if (rc) return rc;
    if ((rc = dev_alloc((void **)&tab->edges, 4))) return rc;
    uint32_t rp[2] = {0, 1}, ed = 0u | (1u << (kSrcBits + 2));
    CP_CUDA_TRY(cudaMemcpy(tab->row_ptr, rp, 8, cudaMemcpyHostToDevice));
    CP_CUDA_TRY(cudaMemcpy(tab->edges, &ed, 4, cudaMemcpyHostToDevice));
    return CP_OK;
}

// Tables of a chain of per-site factors: one per factor, or (paired) one
// two-site table per consecutive pair, the second factor composed after the
// first on every term (an odd one out stays single).  Two chromatic factors
// compose to shifts of at most 3 and coefficients of magnitude at most 5
// (square) or 10 (triangular), so the edges keep a 2-bit shift and take 26 or
// 25 source bits; the build checks both bounds.
static int build_chain(const std::vector<OpDesc> &ops, int paired, int lattice, const RankTables *T_dev,
                       cudaStream_t st, TableSet *ts, std::vector<SiteTable> *out) {
    int rc;
    for (size_t i = 0; i < ops.size();) {
        SiteTable tab;
        if (paired && i + 1 < ops.size()) {
            OpDesc f = ops[i];
            f.fused = 1;
            f.kind_b = ops[i + 1].kind;
            f.i_b = ops[i + 1].i;
            f.out = ops[i + 1].out;
            f.max_terms = ops[i].kind == OP_LAST ? 4 : (lattice == CP_SQUARE ? 16 : 24);
            f.src_bits = lattice == CP_SQUARE ? 26 : 25;
            if ((rc = build_table(f, T_dev, st, &tab))) return rc;
            tab.n_site_out = ops[i].out.size + ops[i + 1].out.size;
            i += 2;
        } else {
            if ((rc = build_table(ops[i], T_dev, st, &tab))) return rc;
            i += 1;
        }
        ts->bytes += (tab.n_dst + 1 + tab.nnz) * 4;
        out->push_back(tab);
    }
    return CP_OK;
}

static int build_tableset(int lattice, int L, int paired, cudaStream_t st, std::shared_ptr<TableSet> *out) {
    const RankTables *T_dev = nullptr;
    RankTables T;
    int rc = device_rank_tables(&T_dev, &T);
    if (rc) return rc;
    auto ts = std::make_shared<TableSet>();
    cudaGetDevice(&ts->device);
    ts->lattice = lattice;
    ts->L = L;
    ts->paired = paired;
    const uint64_t Sb = T.cnt[L];
    const uint64_t Sx = L >= 2 ? T.cnt[L] + T.cnt[L - 1] : Sb;
    ts->S_b = Sb;
    ts->S_max = lattice == CP_SQUARE ? Sx : Sb;
    if (lattice == CP_SQUARE) {
        for (int e = 0; e + 1 < L; ++e) {
            uint32_t *pre = nullptr;
            if ((rc = build_x_prefix(L, e, st, &pre))) return rc;
            ts->x_prefix.push_back(pre);
            ts->bytes += (Sb + 1) * 4;
        }
    }
    std::vector<OpDesc> row_ops, last_ops;
    for (int i = 0; i < L; ++i) {
        OpDesc op{};
        op.m = L;
        op.i = i;
        op.src_bits = (int)kSrcBits;
        if (lattice == CP_SQUARE) {
            op.kind = OP_SQUARE;
            op.max_terms = 4;
            op.in = i == 0 ? Space{SPACE_B, L, 0, 0, Sb, nullptr} : Space{SPACE_X, L, i - 1, 0, Sx, ts->x_prefix[i - 1]};
            op.out = i == L - 1 ? Space{SPACE_B, L, 0, 0, Sb, nullptr} : Space{SPACE_X, L, i, 0, Sx, ts->x_prefix[i]};
        } else {
            op.kind = OP_TRIANGULAR;
            op.max_terms = 8;
            op.in = Space{SPACE_B, L, 0, 0, Sb, nullptr};
            op.out = op.in;
        }
        row_ops.push_back(op);
    }
    for (int i = 0; i + 1 < L; ++i) {  // T_L^last = D_L is the identity on e_0
        OpDesc op{};
        op.kind = OP_LAST;
        op.m = L;
        op.i = i;
        op.src_bits = (int)kSrcBits;
        op.max_terms = 2;
        op.in = Space{SPACE_B, L, 0, 0, T.cnt[L - i], nullptr};
        op.out = Space{SPACE_B, L, 0, 0, T.cnt[L - i - 1], nullptr};
        last_ops.push_back(op);
    }
    if ((rc = build_chain(row_ops, paired, lattice, T_dev, st, ts.get(), &ts->row))) return rc;
    if (L == 1) {
        SiteTable tab;
        if ((rc = identity_table(1, &tab))) return rc;
        ts->last.push_back(tab);
    } else if ((rc = build_chain(last_ops, paired, lattice, T_dev, st, ts.get(), &ts->last))) {
        return rc;
    }
    *out = ts;
    return CP_OK;
}

// Any-v Potts tables on the non-crossing partitions (Catalan space), no projectors.
static int build_potts_tableset(int lattice, int L, int v, cudaStream_t st, std::shared_ptr<TableSet> *out) {
    const RankTables *T_dev = nullptr;
    RankTables T;
    int rc = device_rank_tables(&T_dev, &T);
    if (rc) return rc;
    auto ts = std::make_shared<TableSet>();
    cudaGetDevice(&ts->device);
    ts->lattice = lattice;
    ts->L = L;
    ts->potts = 1;
    ts->v = v;
    const uint64_t S = T.cntc[L];
    ts->src_bits = potts_src_bits(S);
    ts->S_b = ts->S_max = S;
    for (int i = 0; i < L; ++i) {
        OpDesc op{};
        op.kind = lattice == CP_SQUARE ? OP_POTTS_SQUARE : OP_POTTS_TRIANGULAR;
        op.m = L;
        op.i = i;
        op.v = v;
        op.src_bits = ts->src_bits;
        op.max_terms = lattice == CP_SQUARE ? 4 : 8;
        op.in = Space{SPACE_C, L, 0, 0, S, nullptr};
        op.out = op.in;
        SiteTable tab;
        if ((rc = build_table(op, T_dev, st, &tab))) return rc;
        ts->bytes += (tab.n_dst + 1 + tab.nnz) * 4;
        ts->row.push_back(tab);
    }
    if (L == 1) {
        SiteTable tab;
        if ((rc = identity_table(1, &tab))) return rc;
        ts->last.push_back(tab);
    } else {
        for (int i = 0; i + 1 < L; ++i) {  // D_L is the identity on e_0
            OpDesc op{};
            op.kind = OP_POTTS_LAST;
            op.m = L;
            op.i = i;
            op.v = v;
            op.src_bits = ts->src_bits;
            op.max_terms = 2;
            op.in = Space{SPACE_C, L, 0, 0, T.cntc[L - i], nullptr};
            op.out = Space{SPACE_C, L, 0, 0, T.cntc[L - i - 1], nullptr};
            SiteTable tab;
            if ((rc = build_table(op, T_dev, st, &tab))) return rc;
            ts->bytes += (tab.n_dst + 1 + tab.nnz) * 4;
            ts->last.push_back(tab);
        }
    }
    *out = ts;
    return CP_OK;
}

static std::mutex g_cache_mu;
static std::map<std::tuple<int, int, int>, std::shared_ptr<TableSet>> g_cache[64];  // per device
static int g_pairing = 1;  // 0 never, 1 square rows of >= kPairRowBytes, 2 every square table, 3 every table

int factor_pairing() {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    return g_pairing;
}

int set_factor_pairing(int mode) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    const int old = g_pairing;
    g_pairing = mode < 0 ? 0 : (mode > 3 ? 3 : mode);
    return old;
}
static std::map<std::tuple<int, int, int>, std::shared_ptr<TableSet>> g_potts_cache[64];

int get_tables(int lattice, int L, size_t row_bytes, cudaStream_t st, std::shared_ptr<TableSet> *out) {
    int dev = 0;
    CP_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(CP_EINVAL, "device index");
    std::lock_guard<std::mutex> lk(g_cache_mu);
    // Two-site tables halve the vector traffic but not the number of edge copies,
    // which set the pace on narrow rows: they pay on square-lattice rows of a few
    // KB and more; on the triangular lattice a pair has up to 21 terms per source
    // and the gathers ran slower than one factor at a time.
    const int paired = g_pairing == 3 ||
                       (lattice == CP_SQUARE && (g_pairing == 2 || (g_pairing == 1 && row_bytes >= kPairRowBytes)));
    auto key = std::make_tuple(lattice, L, paired);
    auto it = g_cache[dev].find(key);
    if (it != g_cache[dev].end()) {
        *out = it->second;
        return CP_OK;
    }
    std::shared_ptr<TableSet> ts;
    int rc = build_tableset(lattice, L, paired, st, &ts);
    if (rc) return rc;
    g_cache[dev][key] = ts;
    *out = ts;
    return CP_OK;
}

int get_potts_tables(int lattice, int L, int v, cudaStream_t st, std::shared_ptr<TableSet> *out) {
    int dev = 0;
    CP_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(CP_EINVAL, "device index");
    std::lock_guard<std::mutex> lk(g_cache_mu);
    auto key = std::make_tuple(lattice, L, v);
    auto it = g_potts_cache[dev].find(key);
    if (it != g_potts_cache[dev].end()) {
        *out = it->second;
        return CP_OK;
    }
    std::shared_ptr<TableSet> ts;
    int rc = build_potts_tableset(lattice, L, v, st, &ts);
    if (rc) return rc;
    g_potts_cache[dev][key] = ts;
    *out = ts;
    return CP_OK;
}

// Copy one cached (or freshly built) chromatic table to the host.
int debug_table(int lattice, int L, int paired, int which, int index, uint32_t *row_ptr_host, uint64_t max_rows,
                uint32_t *edges_host, uint64_t max_edges, uint64_t info[4]) {
    const int old = set_factor_pairing(paired ? 3 : 0);
    std::shared_ptr<TableSet> ts;
    int rc = get_tables(lattice, L, 0, 0, &ts);
    set_factor_pairing(old);
    if (rc) return rc;
    const std::vector<SiteTable> &v = which ? ts->last : ts->row;
    if (index < 0 || index >= (int)v.size()) return fail(CP_EINVAL, "table index out of range");
    const SiteTable &t = v[index];
    if (info) {
        info[0] = t.n_src;
        info[1] = t.n_dst;
        info[2] = t.nnz;
        info[3] = (uint64_t)t.op.src_bits;
    }
    if (row_ptr_host) {
        if (max_rows < t.n_dst + 1) return fail(CP_EINVAL, "max_rows < n_dst + 1");
        CP_CUDA_TRY(cudaMemcpy(row_ptr_host, t.row_ptr, 4 * (t.n_dst + 1), cudaMemcpyDeviceToHost));
    }
    if (edges_host) {
        if (max_edges < t.nnz) return fail(CP_EINVAL, "max_edges < nnz");
        CP_CUDA_TRY(cudaMemcpy(edges_host, t.edges, 4 * t.nnz, cudaMemcpyDeviceToHost));
    }
    return CP_OK;
}

void clear_table_cache() {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    for (auto &c : g_cache) c.clear();  // strips keep their own shared_ptr alive
    for (auto &c : g_potts_cache) c.clear();
}

static std::mutex g_rt_mu;
static RankTables *g_rt_dev[64];
static RankTables g_rt_host[64];

int device_rank_tables(const RankTables **out_dev, RankTables *host_copy) {
    int dev = 0;
    CP_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(CP_EINVAL, "device index");
    std::lock_guard<std::mutex> lk(g_rt_mu);
    if (!g_rt_dev[dev]) {
        RankTables *p = nullptr;
        int rc = dev_alloc((void **)&p, sizeof(RankTables));
        if (rc) return rc;
        rank_tables_kernel<<<1, 32>>>(p);
        CP_CUDA_TRY(cudaGetLastError());
        CP_CUDA_TRY(cudaMemcpy(&g_rt_host[dev], p, sizeof(RankTables), cudaMemcpyDeviceToHost));
        g_rt_dev[dev] = p;
    }
    *out_dev = g_rt_dev[dev];
    if (host_copy) *host_copy = g_rt_host[dev];
    return CP_OK;
}

// ------------------------------------------------------------------ debug: rank/unrank sweep

__global__ void check_space_kernel(Space sp, const RankTables *Tg, unsigned long long *bad) {
    __shared__ RankTables T;
    stage_tables(T, Tg);
    uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= sp.size) return;
    Labels s;
    space_unrank(r, sp, s, T);
    Labels c = s;
    canonicalise(c, sp.m);
    bool ok = space_contains(s, sp) && space_rank(s, sp, T) == r;
    for (int i = 0; i < sp.m; ++i) ok = ok && c.v[i] == s.v[i];
    if (!ok) atomicAdd(bad, 1ull);
}

int check_space(int kind, int m, int e, uint64_t *n_bad, uint64_t *size) {
    const RankTables *T_dev = nullptr;
    RankTables T;
    int rc = device_rank_tables(&T_dev, &T);
    if (rc) return rc;
    Space sp{kind, m, e, 0, kind == SPACE_X ? T.cnt[m] + T.cnt[m - 1] : (kind == SPACE_C ? T.cntc[m] : T.cnt[m]),
             nullptr};
    uint32_t *pre = nullptr;
    if (kind == SPACE_X && (rc = build_x_prefix(m, e, 0, &pre))) return rc;
    sp.prefix = pre;
    unsigned long long *bad = nullptr;
    if ((rc = dev_alloc((void **)&bad, 8))) {
        dev_free(pre);
        return rc;
    }
    CP_CUDA_TRY(cudaMemset(bad, 0, 8));
    check_space_kernel<<<(unsigned)((sp.size + 127) / 128), 128>>>(sp, T_dev, bad);
    CP_CUDA_TRY(cudaGetLastError());
    unsigned long long h = 0;
    CP_CUDA_TRY(cudaMemcpy(&h, bad, 8, cudaMemcpyDeviceToHost));
    dev_free(bad);
    dev_free(pre);
    *n_bad = h;
    *size = sp.size;
    return CP_OK;
}

// Copy the ranked partitions of a space to the host (labels, m bytes each).
__global__ void enumerate_kernel(Space sp, const RankTables *Tg, uint8_t *out) {
    __shared__ RankTables T;
    stage_tables(T, Tg);
    uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= sp.size) return;
    Labels s;
    space_unrank(r, sp, s, T);
    for (int i = 0; i < sp.m; ++i) out[r * sp.m + i] = s.v[i];
}

int enumerate_space(int kind, int m, int e, uint8_t *out_host, uint64_t max_states, uint64_t *size) {
    const RankTables *T_dev = nullptr;
    RankTables T;
    int rc = device_rank_tables(&T_dev, &T);
    if (rc) return rc;
    Space sp{kind, m, e, 0, kind == SPACE_X ? T.cnt[m] + T.cnt[m - 1] : (kind == SPACE_C ? T.cntc[m] : T.cnt[m]),
             nullptr};
    *size = sp.size;
    if (sp.size > max_states) return fail(CP_EINVAL, "output buffer too small");
    uint32_t *pre = nullptr;
    if (kind == SPACE_X && (rc = build_x_prefix(m, e, 0, &pre))) return rc;
    sp.prefix = pre;
    uint8_t *d = nullptr;
    if ((rc = dev_alloc((void **)&d, sp.size * m))) {
        dev_free(pre);
        return rc;
    }
    enumerate_kernel<<<(unsigned)((sp.size + 127) / 128), 128>>>(sp, T_dev, d);
    CP_CUDA_TRY(cudaGetLastError());
    CP_CUDA_TRY(cudaMemcpy(out_host, d, sp.size * m, cudaMemcpyDeviceToHost));
    dev_free(d);
    dev_free(pre);
    return CP_OK;
}

}  // namespace cp
