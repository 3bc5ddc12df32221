// Device code for the connectivity states of the top row (Sec. 3.1-3.4):
// label arrays, the single-edge operators, and the rank/unrank bijection of
// the NCNNN partitions and of the square lattice's excepted spaces.
#pragma once

#include <stdint.h>

#include "cp_internal.h"

namespace cp {

constexpr int kMaxL = CP_MAX_L;
constexpr uint8_t kFresh = 31;  // temporary label of a detached site (labels are < kMaxL)

// A partition of the sites 0..m-1: block labels in first-occurrence order.
struct Labels {
    uint8_t v[kMaxL];
};

__device__ __forceinline__ void canonicalise(Labels &s, int m) {
    uint8_t map[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) map[k] = 0xFF;
    uint8_t next = 0;
    for (int i = 0; i < m; ++i) {
        uint8_t x = s.v[i];
        if (map[x] == 0xFF) map[x] = next++;
        s.v[i] = map[x];
    }
}

// J_{a,b} for a !~ b: merge the two blocks (the factor w is the caller's shift).
__device__ __forceinline__ void join_blocks(Labels &s, int m, int a, int b) {
    uint8_t la = s.v[a], lb = s.v[b];
    for (int i = 0; i < m; ++i)
        if (s.v[i] == lb) s.v[i] = la;
    canonicalise(s, m);
}

// D_i: site i becomes a singleton.
__device__ __forceinline__ void detach_site(Labels &s, int m, int i) {
    s.v[i] = kFresh;
    canonicalise(s, m);
}

// Non-crossing test in O(m): scanning left to right, a block that reappears
// must be the innermost open one.
__device__ __forceinline__ bool is_noncrossing(const Labels &s, int m) {
    int8_t last[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) last[k] = -1;
    for (int i = 0; i < m; ++i) last[s.v[i]] = (int8_t)i;
    uint8_t stack[kMaxL];
    int sp = 0;
    uint32_t open = 0;  // bit set of open labels
    for (int i = 0; i < m; ++i) {
        uint8_t b = s.v[i];
        if (open >> b & 1u) {
            if (sp == 0 || stack[sp - 1] != b) return false;
            if (last[b] == i) { --sp; open &= ~(1u << b); }
        } else if (last[b] != i) {
            stack[sp++] = b;
            open |= 1u << b;
        }
    }
    return true;
}

// Neighbour rule: no (j, j+1) in one block, except the pair j == skip.
__device__ __forceinline__ bool nn_ok(const Labels &s, int m, int skip) {
    for (int j = 0; j + 1 < m; ++j)
        if (j != skip && s.v[j] == s.v[j + 1]) return false;
    return true;
}

// Rank of an NCNNN partition of the points lo..hi-1 in the paper's order
// (Sec. 3.4): a point alone first (rank of the rest), then by the smallest
// partner lo+2+k of point lo, inner points as the most significant digit and
// the right part (from the partner on) as the least significant one.
// Returns ~0ull if the partition violates the neighbour rule at the first point.
__device__ __forceinline__ uint64_t ncnnn_rank(const Labels &s, int lo, int hi, const RankTables &T) {
    int sa[kMaxL + 1], sb[kMaxL + 1];
    uint64_t smul[kMaxL + 1];
    int sp = 0;
    uint64_t r = 0;
    int a = lo, b = hi;
    uint64_t mu = 1;
    for (;;) {
        while (b - a > 2) {
            int n = b - a;
            if (s.v[a + 1] == s.v[a]) return ~0ull;
            int j = -1;
            for (int t = a + 2; t < b; ++t)
                if (s.v[t] == s.v[a]) { j = t; break; }
            if (j < 0) { ++a; continue; }
            int k = j - a - 2;
            uint64_t cr = T.cnt[b - j];
            r += mu * T.off[n * kTblStride + k];
            sa[sp] = a + 1; sb[sp] = j; smul[sp] = mu * cr; ++sp;   // inner part, later
            a = j;                                                   // right part, now
        }
        if (b - a == 2 && s.v[a] == s.v[a + 1]) return ~0ull;
        if (sp == 0) break;
        --sp;
        a = sa[sp]; b = sb[sp]; mu = smul[sp];
    }
    return r;
}

// Inverse of ncnnn_rank on points lo..hi-1; labels are assigned in
// first-occurrence order, so the result is canonical when lo == 0.
__device__ __forceinline__ void ncnnn_unrank(uint64_t r, int lo, int hi, Labels &s, const RankTables &T) {
    for (int i = lo; i < hi; ++i) s.v[i] = 0xFF;
    uint8_t next = 0;
    int sa[kMaxL + 1], sb[kMaxL + 1];
    uint64_t sr[kMaxL + 1];
    int sp = 0;
    int a = lo, b = hi;
    for (;;) {
        while (b - a >= 1) {
            if (s.v[a] == 0xFF) s.v[a] = next++;
            int n = b - a;
            if (n <= 2) {
                if (n == 2) s.v[a + 1] = next++;
                break;
            }
            if (r < T.cnt[n - 1]) { ++a; continue; }   // point a alone
            int k = 0;
            while (k + 1 <= n - 3 && T.off[n * kTblStride + k + 1] <= r) ++k;
            r -= T.off[n * kTblStride + k];
            uint64_t cr = T.cnt[n - k - 2];
            uint64_t inner = r / cr, right = r - inner * cr;
            int j = a + 2 + k;
            s.v[j] = s.v[a];
            sa[sp] = j; sb[sp] = b; sr[sp] = right; ++sp;   // right part after the inner one
            a = a + 1; b = j; r = inner;
        }
        if (sp == 0) break;
        --sp;
        a = sa[sp]; b = sb[sp]; r = sr[sp];
    }
}

// Rank of a non-crossing partition of points lo..hi-1: the first point alone
// first (rank of the rest), then by its smallest partner lo+1+k, inner points
// as the most significant digit and the right part (from the partner on) as
// the least significant one.  The count recursion is Catalan's.
__device__ __forceinline__ uint64_t nc_rank(const Labels &s, int lo, int hi, const RankTables &T) {
    int sa[kMaxL + 1], sb[kMaxL + 1];
    uint64_t smul[kMaxL + 1];
    int sp = 0;
    uint64_t r = 0;
    int a = lo, b = hi;
    uint64_t mu = 1;
    for (;;) {
        while (b - a > 1) {
            int n = b - a, j = -1;
            for (int t = a + 1; t < b; ++t)
                if (s.v[t] == s.v[a]) { j = t; break; }
            if (j < 0) { ++a; continue; }
            int k = j - a - 1;
            r += mu * T.offc[n * kTblStride + k];
            sa[sp] = a + 1; sb[sp] = j; smul[sp] = mu * T.cntc[b - j]; ++sp;  // inner part, later
            a = j;                                                              // right part, now
        }
        if (sp == 0) break;
        --sp;
        a = sa[sp]; b = sb[sp]; mu = smul[sp];
    }
    return r;
}

__device__ __forceinline__ void nc_unrank(uint64_t r, int lo, int hi, Labels &s, const RankTables &T) {
    for (int i = lo; i < hi; ++i) s.v[i] = 0xFF;
    uint8_t next = 0;
    int sa[kMaxL + 1], sb[kMaxL + 1];
    uint64_t sr[kMaxL + 1];
    int sp = 0;
    int a = lo, b = hi;
    for (;;) {
        while (b - a >= 1) {
            if (s.v[a] == 0xFF) s.v[a] = next++;
            int n = b - a;
            if (n == 1) break;
            if (r < T.cntc[n - 1]) { ++a; continue; }  // point a alone
            int k = 0;
            while (k + 1 <= n - 2 && T.offc[n * kTblStride + k + 1] <= r) ++k;
            r -= T.offc[n * kTblStride + k];
            uint64_t cr = T.cntc[n - 1 - k];
            uint64_t inner = r / cr, right = r - inner * cr;
            int j = a + 1 + k;
            s.v[j] = s.v[a];
            sa[sp] = j; sb[sp] = b; sr[sp] = right; ++sp;  // right part after the inner one
            a = a + 1; b = j; r = inner;
        }
        if (sp == 0) break;
        --sp;
        a = sa[sp]; b = sb[sp]; r = sr[sp];
    }
}

// Rank in a space (SPACE_B: the paper's order; SPACE_X: the interleaved order,
// see Space).  Returns ~0ull for a partition outside the space's rule.
__device__ __forceinline__ uint64_t space_rank(const Labels &s, const Space &sp, const RankTables &T) {
    const int m = sp.m;
    if (sp.kind == SPACE_X) {
        const int e = sp.e;
        if (s.v[e] == s.v[e + 1]) {
            Labels t = s;
            detach_site(t, m, e);
            uint64_t b = ncnnn_rank(t, 0, m, T);
            return b == ~0ull ? b : b + sp.prefix[b] + 1;
        }
        uint64_t b = ncnnn_rank(s, 0, m, T);
        return b == ~0ull ? b : b + sp.prefix[b];
    }
    if (sp.kind == SPACE_C) return nc_rank(s, 0, m, T);
    return ncnnn_rank(s, 0, m, T);
}

__device__ __forceinline__ void space_unrank(uint64_t r, const Space &sp, Labels &s, const RankTables &T) {
    const int m = sp.m;
    if (sp.kind == SPACE_X) {
        // largest b with b + prefix[b] <= r (strictly increasing in b)
        uint64_t lo = 0, hi = T.cnt[m] - 1;
        while (lo < hi) {
            uint64_t mid = (lo + hi + 1) >> 1;
            if (mid + sp.prefix[mid] <= r) lo = mid; else hi = mid - 1;
        }
        ncnnn_unrank(lo, 0, m, s, T);
        if (r != lo + sp.prefix[lo]) join_blocks(s, m, sp.e, sp.e + 1);
        return;
    }
    if (sp.kind == SPACE_C) {
        nc_unrank(r, 0, m, s, T);
        return;
    }
    ncnnn_unrank(r, 0, m, s, T);
}

// Membership test of a canonical partition in a space (debug/validation).
__device__ __forceinline__ bool space_contains(const Labels &s, const Space &sp) {
    if (sp.kind == SPACE_C) return is_noncrossing(s, sp.m);
    return is_noncrossing(s, sp.m) && nn_ok(s, sp.m, sp.kind == SPACE_X ? sp.e : -1);
}

// Stage the rank tables into shared memory (all threads of the block call).
__device__ __forceinline__ void stage_tables(RankTables &dst, const RankTables *src) {
    const uint64_t *a = reinterpret_cast<const uint64_t *>(src);
    uint64_t *b = reinterpret_cast<uint64_t *>(&dst);
    for (int k = threadIdx.x; k < (int)(sizeof(RankTables) / 8); k += blockDim.x) b[k] = a[k];
    __syncthreads();
}

}  // namespace cp
