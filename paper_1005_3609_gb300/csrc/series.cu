// Finite-lattice combination of the rectangles into the bulk, surface and
// corner series, modulo each prime (Sec. 4.1-4.3).
//
// f_x = sum_{(r,s) in B(k)} weight_x(r,s) log P~_{r,s}, eqs. (fb)-(fc), with
// P~ written in z (w = z/(1+z), eq. (def_z)) on the square lattice and in x
// (w = -x/(1-x)^2, q = 2 - x - 1/x) on the triangular one.  Each P~ has
// constant term 1, so log and exp are power series with denominators up to
// n < p: everything is exact modulo p.  Output per prime:
//   series 0: square sum alpha_k z^k = (1+z)^2 exp(f_b - log q)   (Table 1)
//             triangular (1-x)^2 exp(f_b - log q)   (= Baxter's product, eq. (efb))
//   series 1: exp(f_s);  series 2: exp(f_c).
// For the square lattice at odd k the extra term mu_{2m} z^{4m-1}, m = (k-1)/2,
// is added to f_b and -m mu_{2m} z^{4m-1} to f_s (Sec. 4.2), which extends the
// bulk and surface series by one term.
#include <cuda_runtime.h>

#include "cp_internal.h"
#include "series.h"

namespace cp {

// Arithmetic modulo a prime p < 2^31.  Products use Barrett reduction with
// m = floor((2^64 - 1) / p): q = floor(x m / 2^64) undershoots floor(x / p) by at
// most 2 for x < 2^62, so x - q p < 3p needs at most two subtractions.
struct Mod {
    uint32_t p;
    uint64_t m;
};
__device__ __forceinline__ Mod make_mod(uint32_t p) { return Mod{p, 0xFFFFFFFFFFFFFFFFull / p}; }
__device__ __forceinline__ uint32_t mm(uint32_t a, uint32_t b, const Mod &M) {
    const uint64_t x = (uint64_t)a * b;
    uint64_t r = x - __umul64hi(x, M.m) * M.p;
    if (r >= M.p) r -= M.p;
    if (r >= M.p) r -= M.p;
    return (uint32_t)r;
}
__device__ __forceinline__ uint32_t ad(uint32_t a, uint32_t b, uint32_t p) {
    uint32_t t = a + b;
    return t >= p ? t - p : t;
}
__device__ __forceinline__ uint32_t sb(uint32_t a, uint32_t b, uint32_t p) { return a >= b ? a - b : a + p - b; }
__device__ __forceinline__ uint32_t from_int(long long v, uint32_t p) {
    long long r = v % (long long)p;
    return (uint32_t)(r < 0 ? r + p : r);
}
__device__ uint32_t pw(uint32_t a, uint32_t e, const Mod &M) {
    uint32_t r = 1;
    while (e) {
        if (e & 1) r = mm(r, a, M);
        a = mm(a, a, M);
        e >>= 1;
    }
    return r;
}

// Finite-lattice weights (Sec. 4.1); beta with (r+s+2)/2 on delta_{r+s,k-3}
// (the printed (r+s-2)/2 violates the sum rules), all integers.
__device__ long long flm_weight(int which, int k, int r, int s) {
    const int t = r + s;
    const long long f = (r == s) ? 1 : 2;
    if (which == 0) {
        int c = t == k ? 1 : t == k - 1 ? -3 : t == k - 2 ? 3 : t == k - 3 ? -1 : 0;
        return f * c;
    }
    if (which == 1) {  // (2 - delta) * num / 2, num even whenever r == s
        long long num = t == k ? (2 - t) : t == k - 1 ? (3 * t - 2) : t == k - 2 ? -(3 * t + 2) : t == k - 3 ? (t + 2) : 0;
        return f * num / 2;
    }
    long long rs = (long long)r * s;
    long long c = t == k ? (long long)(r - 1) * (s - 1) : t == k - 1 ? (1 + t - 3 * rs)
                : t == k - 2 ? (3 * rs + t - 1) : t == k - 3 ? -(long long)(r + 1) * (s + 1) : 0;
    return f * c;
}

// mu_{2m} mod p from sum_{p>=4} mu_p y^p = y^4 (2-2y-y sqrt(1-4y)) / ((1-4y)(2+y))
//                                        + y^6 (3-4y-4 sqrt(1-4y)) / (1-4y)^2      (y = x^2)
__device__ uint32_t mu_mod(int idx, const Mod &M) {
    const uint32_t p = M.p;
    const int n = idx + 1;
    uint32_t sq[kMaxSeries], g1[kMaxSeries], q1[kMaxSeries], t1[kMaxSeries], t2[kMaxSeries];
    // sqrt(1-4y) = 1 - 2 sum_{j>=1} C_{j-1} y^j, Catalan C_j = C_{j-1} 2(2j-1)/(j+1)
    uint32_t cat = 1;
    sq[0] = 1;
    for (int j = 1; j < n; ++j) {
        sq[j] = sb(0, mm(2, cat, M), p);
        cat = mm(mm(cat, from_int(2 * (2 * j - 1), p), M), pw(j + 1, p - 2, M), M);
    }
    const uint32_t inv2 = pw(2, p - 2, M);
    for (int j = 0; j < n; ++j) {
        g1[j] = pw(4, j, M);                                    // 1/(1-4y)
        q1[j] = mm(j & 1 ? p - 1 : 1, pw(inv2, j + 1, M), M);   // 1/(2+y)
    }
    // numerators
    uint32_t a[kMaxSeries], b[kMaxSeries];
    for (int j = 0; j < n; ++j) {
        a[j] = (j == 0 ? 2 : 0);
        if (j == 1) a[j] = sb(a[j], 2, p);
        if (j >= 1) a[j] = sb(a[j], sq[j - 1], p);
        b[j] = (j == 0 ? 3 : 0);
        if (j == 1) b[j] = sb(b[j], 4, p);
        b[j] = sb(b[j], mm(4, sq[j], M), p);
    }
    for (int j = 0; j < n; ++j) {  // t1 = a * g1 * q1, t2 = b * g1 * g1
        uint32_t x = 0, y = 0;
        for (int i = 0; i <= j; ++i) {
            x = ad(x, mm(a[i], g1[j - i], M), p);
            y = ad(y, mm(g1[i], g1[j - i], M), p);
        }
        t1[j] = x;
        t2[j] = y;
    }
    uint32_t u = 0, v = 0;
    if (idx >= 4) {
        int j = idx - 4;
        for (int i = 0; i <= j; ++i) u = ad(u, mm(t1[i], q1[j - i], M), p);
    }
    if (idx >= 6) {
        int j = idx - 6;
        for (int i = 0; i <= j; ++i) v = ad(v, mm(b[i], t2[j - i], M), p);
    }
    return ad(u, v, p);
}

// One block per prime.  Shared: logs[n_rects][n], the inverses 1/i (i < n) and
// the three weighted sums; one thread per rectangle for its substitution and
// logarithm, then one thread per coefficient for the weighted sums, then one
// warp per series for the exponential (the sum of each step spread over the
// lanes).
__global__ void flm_series_kernel(const uint32_t *__restrict__ ptilde, const int2 *__restrict__ rects,
                                  const uint32_t *__restrict__ primes, SeriesParams sp, uint32_t *__restrict__ out,
                                  int *err) {
    extern __shared__ uint32_t logs[];
    __shared__ uint32_t inv[kMaxSeries];
    __shared__ uint32_t acc[3][kMaxSeries];
    __shared__ uint32_t E[3][kMaxSeries];
    const int pi = blockIdx.x;
    const uint32_t p = primes[pi];
    const Mod M = make_mod(p);
    const int n = sp.n, D1 = sp.D1, P = sp.P;
    for (int i = threadIdx.x; i < n; i += blockDim.x) inv[i] = i ? pw((uint32_t)i, p - 2, M) : 0u;
    __syncthreads();
    for (int j = threadIdx.x; j < sp.n_rects; j += blockDim.x) {
        uint32_t f[kMaxSeries], h[kMaxSeries];
        const int grp = pi / sp.Pg, pk = pi - grp * sp.Pg;
        const uint32_t *src = ptilde + ((size_t)grp * sp.n_rects + j) * D1 * sp.Pg;
        for (int i = 0; i < n; ++i) f[i] = 0;
        // Horner: f = P~(w(t)) mod t^n, multiplying by w(t) with its recurrence
        for (int d = min(D1 - 1, n - 1); d >= 0; --d) {
            if (sp.lattice == CP_SQUARE) {  // * z/(1+z):  y_i = f_{i-1} - y_{i-1}
                uint32_t prev = 0;
                for (int i = 0; i < n; ++i) {
                    uint32_t s = i ? f[i - 1] : 0;
                    uint32_t y = sb(s, prev, p);
                    h[i] = y;
                    prev = y;
                }
            } else {  // * -x/(1-x)^2: shift, two prefix sums, negate
                uint32_t u = 0, v = 0;
                for (int i = 0; i < n; ++i) {
                    uint32_t s = i ? f[i - 1] : 0;
                    u = ad(u, s, p);
                    v = ad(v, u, p);
                    h[i] = sb(0, v, p);
                }
            }
            for (int i = 0; i < n; ++i) f[i] = h[i];
            f[0] = ad(f[0], src[(size_t)d * sp.Pg + pk], p);
        }
        if (f[0] != 1) atomicOr(err, 1);
        // log f: h = f'/f, g_i = h_{i-1}/i
        for (int i = 0; i + 1 < n; ++i) {
            uint32_t a = mm(f[i + 1], (uint32_t)(i + 1), M);
            for (int q = 1; q <= i; ++q) a = sb(a, mm(f[q], h[i - q], M), p);
            h[i] = a;
        }
        uint32_t *g = logs + (size_t)j * n;
        g[0] = 0;
        for (int i = 1; i < n; ++i) g[i] = mm(h[i - 1], inv[i], M);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        uint32_t a0 = 0, a1 = 0, a2 = 0;
        for (int j = 0; j < sp.n_rects; ++j) {
            const int r = rects[j].x, s = rects[j].y;
            uint32_t g = logs[(size_t)j * n + i];
            a0 = ad(a0, mm(from_int(flm_weight(0, sp.k, r, s), p), g, M), p);
            a1 = ad(a1, mm(from_int(flm_weight(1, sp.k, r, s), p), g, M), p);
            a2 = ad(a2, mm(from_int(flm_weight(2, sp.k, r, s), p), g, M), p);
        }
        acc[0][i] = a0;
        acc[1][i] = a1;
        acc[2][i] = a2;
    }
    __syncthreads();
    // E = exp(a): E_0 = 1, i E_i = sum_{q=1..i} q a_q E_{i-q}; warp x for series x
    const int x = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (x < 3) {
        if (lane == 0) E[x][0] = 1;
        __syncwarp();
        for (int i = 1; i < n; ++i) {
            uint32_t s = 0;
            for (int q = 1 + lane; q <= i; q += 32) s = ad(s, mm(mm((uint32_t)q, acc[x][q], M), E[x][i - q], M), p);
            for (int o = 16; o > 0; o >>= 1) s = ad(s, __shfl_xor_sync(0xffffffffu, s, o), p);
            if (lane == 0) E[x][i] = mm(s, inv[i], M);
            __syncwarp();
        }
        if (lane == 0) {
            uint32_t *o = out + ((size_t)x * P + pi) * n;
            if (x == 0) {
                const bool sq = sp.lattice == CP_SQUARE;
                for (int i = 0; i < n; ++i) {  // (1 +- t)^2 E
                    uint32_t v = E[x][i];
                    if (i >= 1) v = sq ? ad(v, mm(2, E[x][i - 1], M), p) : sb(v, mm(2, E[x][i - 1], M), p);
                    if (i >= 2) v = ad(v, E[x][i - 2], p);
                    o[i] = v;
                }
            } else {
                for (int i = 0; i < n; ++i) o[i] = E[x][i];
            }
            if (sp.add_mu && x < 2) {  // first-order: exp(f + c t^{n-1}) = exp(f) (1 + c t^{n-1}) mod t^n
                const uint32_t mu = mu_mod(2 * sp.mmax, M);
                const uint32_t c = x == 0 ? mu : sb(0, mm((uint32_t)sp.mmax, mu, M), p);
                o[n - 1] = ad(o[n - 1], c, p);  // series 0 and 1 start with 1
            }
        }
    }
}

int launch_flm_series(const uint32_t *ptilde, const int2 *rects, const uint32_t *primes, const SeriesParams &sp,
                      uint32_t *out, int *err, cudaStream_t st) {
    size_t shm = (size_t)sp.n_rects * sp.n * 4;
    if (shm > 200 * 1024) return fail(CP_EINVAL, "too many rectangles for the series kernel");
    if (shm > 48 * 1024)
        CP_CUDA_TRY(cudaFuncSetAttribute(flm_series_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    flm_series_kernel<<<sp.P, 96, shm, st>>>(ptilde, rects, primes, sp, out, err);  // 3 warps: one per series
    CP_CUDA_TRY(cudaGetLastError());
    return CP_OK;
}

}  // namespace cp
