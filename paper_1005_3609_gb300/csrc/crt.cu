// Chinese remaindering of the residues (Sec. 3.5) and the prime set.
//
// Garner's mixed-radix form x = v_0 + v_1 p_0 + v_2 p_0 p_1 + ..., one thread
// per coefficient, then Horner in 32-bit limbs and the symmetric
// representative in (-prod/2, prod/2] as two's complement.
//
// The paper adds primes until the recombined result stops changing.  The
// checked variants report, per coefficient, whether (bit 1) the value
// recombined from the first n-1 primes differs from the one from all n, and
// (bit 0) whether a caller-given bound |c| < 2^bits is not covered, i.e.
// bits + 2 > bit length of the prime product (covered means 2 |c| < prod, the
// range the symmetric representative recovers).
#include <cuda_runtime.h>

#include <mutex>
#include <string>
#include <vector>

#include "cp_internal.h"

namespace cp {

constexpr int kMaxLimbs = 64;

__device__ __forceinline__ uint32_t mulmod(uint32_t a, uint32_t b, uint32_t p) {
    return (uint32_t)(((uint64_t)a * b) % p);
}

__device__ uint32_t powmod(uint32_t a, uint32_t e, uint32_t p) {
    uint32_t r = 1 % p;
    while (e) {
        if (e & 1) r = mulmod(r, a, p);
        a = mulmod(a, a, p);
        e >>= 1;
    }
    return r;
}

struct CrtParams {
    uint32_t primes[CP_MAX_PRIMES];
    int n_primes, n_coeffs, limbs;
    int prod_bits;  // bit length of the product of all primes
};

// Symmetric representative of the mixed-radix digits v_0..v_{k-1} (primes
// p_0..p_{k-1}) in n two's-complement limbs: x = sum v_i prod_{j<i} p_j, minus
// prod_{j<k} p_j when 2x exceeds it.
__device__ void crt_symmetric(const uint32_t *v, const uint32_t *primes, int k, int n, uint32_t *x) {
    uint32_t M[kMaxLimbs];
    for (int l = 0; l < n; ++l) x[l] = M[l] = 0;
    x[0] = v[k - 1];
    M[0] = 1;
    for (int i = k - 2; i >= 0; --i) {  // x = x * p_i + v_i
        uint64_t carry = v[i];
        for (int l = 0; l < n; ++l) {
            uint64_t y = (uint64_t)x[l] * primes[i] + carry;
            x[l] = (uint32_t)y;
            carry = y >> 32;
        }
    }
    for (int i = 0; i < k; ++i) {  // M = prod p_i
        uint64_t carry = 0;
        for (int l = 0; l < n; ++l) {
            uint64_t y = (uint64_t)M[l] * primes[i] + carry;
            M[l] = (uint32_t)y;
            carry = y >> 32;
        }
    }
    // if 2x > M: x -= M (two's complement wraps to the negative value)
    // 2x has limbs (x[l] << 1) | (x[l-1] >> 31) plus the bit x[n-1] >> 31 above the top limb
    int cmp = (x[n - 1] >> 31) ? 1 : 0;
    for (int l = n - 1; l >= 0 && cmp == 0; --l) {
        uint32_t y = (x[l] << 1) | (l > 0 ? x[l - 1] >> 31 : 0u);
        if (y != M[l]) cmp = y > M[l] ? 1 : -1;
    }
    if (cmp > 0) {
        uint64_t borrow = 0;
        for (int l = 0; l < n; ++l) {
            uint64_t y = (uint64_t)x[l] - M[l] - borrow;
            x[l] = (uint32_t)y;
            borrow = (y >> 63) & 1;
        }
    }
}

// inv[i*P + j] = p_j^{-1} mod p_i (j < i), by Fermat's little theorem.
// flags (optional): per coefficient, bit 0 = bound not covered (bound_bits given),
// bit 1 = the first P-1 primes give another value (always set for P = 1).
__global__ void crt_kernel(const uint32_t *__restrict__ res, uint32_t *__restrict__ limbs_out, CrtParams cp_,
                           const uint32_t *__restrict__ bound_bits, uint32_t *__restrict__ flags) {
    __shared__ uint32_t inv[CP_MAX_PRIMES * CP_MAX_PRIMES];
    const int P = cp_.n_primes;
    for (int k = threadIdx.x; k < P * P; k += blockDim.x) {
        int i = k / P, j = k % P;
        inv[k] = j < i ? powmod(cp_.primes[j] % cp_.primes[i], cp_.primes[i] - 2, cp_.primes[i]) : 0;
    }
    __syncthreads();
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cp_.n_coeffs) return;
    uint32_t v[CP_MAX_PRIMES];
    for (int i = 0; i < P; ++i) {
        const uint32_t pi = cp_.primes[i];
        uint32_t t = res[(size_t)i * cp_.n_coeffs + c] % pi;
        for (int j = 0; j < i; ++j) {
            uint32_t vj = v[j] % pi;
            t = t >= vj ? t - vj : t + pi - vj;
            t = mulmod(t, inv[i * P + j], pi);
        }
        v[i] = t;
    }
    const int n = cp_.limbs;
    uint32_t x[kMaxLimbs];
    crt_symmetric(v, cp_.primes, P, n, x);
    for (int l = 0; l < n; ++l) limbs_out[(size_t)c * n + l] = x[l];
    if (!flags) return;
    uint32_t f = 0;
    if (bound_bits && (int)bound_bits[c] + 2 > cp_.prod_bits) f |= 1u;
    if (P < 2) {
        f |= 2u;
    } else {
        uint32_t y[kMaxLimbs];
        crt_symmetric(v, cp_.primes, P - 1, n, y);
        for (int l = 0; l < n; ++l)
            if (y[l] != x[l]) f |= 2u;
    }
    flags[c] = f;
}

// Bit length of the product of the primes, exactly (multi-limb product).
int primes_product_bits(const uint32_t *primes, int P) {
    std::vector<uint32_t> x(1, 1u);
    for (int k = 0; k < P; ++k) {
        uint64_t carry = 0;
        for (auto &l : x) {
            const uint64_t y = (uint64_t)l * primes[k] + carry;
            l = (uint32_t)y;
            carry = y >> 32;
        }
        if (carry) x.push_back((uint32_t)carry);
    }
    int bits = 32 * ((int)x.size() - 1);
    for (uint32_t top = x.back(); top; top >>= 1) ++bits;
    return bits;
}

static int crt_params(const uint32_t *primes, int P, int n_coeffs, int limbs, CrtParams *cp_) {
    int rc = check_primes(primes, P);
    if (rc) return rc;
    if (n_coeffs < 0) return fail(CP_EINVAL, "n_coeffs < 0");
    if (limbs < 1 || limbs > kMaxLimbs) return fail(CP_EINVAL, "limbs_per_coeff must be 1..64");
    const int bits = primes_product_bits(primes, P);
    if (limbs * 32 < bits + 1)
        return fail(CP_EINVAL, "limbs_per_coeff * 32 must be at least the bit length of the prime product (" +
                                   std::to_string(bits) + ") plus 1");
    for (int k = 0; k < P; ++k) cp_->primes[k] = primes[k];
    cp_->n_primes = P;
    cp_->n_coeffs = n_coeffs;
    cp_->limbs = limbs;
    cp_->prod_bits = bits;
    return CP_OK;
}

// Device CRT with optional checks (bound_dev may be NULL; flags_dev NULL = no checks).
int launch_crt(const uint32_t *res_dev, const uint32_t *primes, int P, int n_coeffs, uint32_t *limbs_dev, int limbs,
               const uint32_t *bound_dev, uint32_t *flags_dev, cudaStream_t st) {
    CrtParams prm{};
    int rc = crt_params(primes, P, n_coeffs, limbs, &prm);
    if (rc) return rc;
    if (n_coeffs == 0) return CP_OK;
    crt_kernel<<<(n_coeffs + 63) / 64, 64, 0, st>>>(res_dev, limbs_dev, prm, bound_dev, flags_dev);
    CP_CUDA_TRY(cudaGetLastError());
    return CP_OK;
}

// Bit lengths of C(n_edges, j), j < n_coeffs (Whitney's bound on |c_j|), exactly.
void binomial_bits(uint64_t n_edges, int n_coeffs, uint32_t *bits_out) {
    std::vector<uint32_t> b(1, 1u);  // C(n, 0) = 1, little-endian limbs
    for (int j = 0; j < n_coeffs; ++j) {
        if (b.size() == 1 && b[0] == 0) {
            bits_out[j] = 0;
            continue;
        }
        uint32_t bits = 32 * (uint32_t)(b.size() - 1);
        for (uint32_t top = b.back(); top; top >>= 1) ++bits;
        bits_out[j] = bits;
        // C(n, j+1) = C(n, j) (n - j) / (j + 1), exact
        const uint64_t mul = (uint64_t)j < n_edges ? n_edges - (uint64_t)j : 0;
        uint64_t carry = 0;
        for (auto &l : b) {
            const unsigned __int128 y = (unsigned __int128)l * mul + carry;
            l = (uint32_t)y;
            carry = (uint64_t)(y >> 32);
        }
        while (carry) {
            b.push_back((uint32_t)carry);
            carry >>= 32;
        }
        const uint64_t div = (uint64_t)j + 1;
        unsigned __int128 rem = 0;
        for (size_t i = b.size(); i-- > 0;) {
            const unsigned __int128 cur = (rem << 32) | b[i];
            b[i] = (uint32_t)(cur / div);
            rem = cur % div;
        }
        while (b.size() > 1 && b.back() == 0) b.pop_back();
    }
}

uint64_t rectangle_edges(int lattice, int L, int N) {
    uint64_t e = (uint64_t)L * (N - 1) + (uint64_t)N * (L - 1);
    if (lattice == CP_TRIANGULAR) e += (uint64_t)(L - 1) * (N - 1);
    return e;
}

}  // namespace cp

using namespace cp;

extern "C" int cp_crt_device(const uint32_t *res_dev, const uint32_t *primes, int P, int n_coeffs, uint32_t *limbs_dev,
                             int limbs, void *stream) {
    if (n_coeffs > 0 && (!res_dev || !limbs_dev)) return fail(CP_EINVAL, "NULL argument");
    return launch_crt(res_dev, primes, P, n_coeffs, limbs_dev, limbs, nullptr, nullptr, (cudaStream_t)stream);
}

// Host-buffer CRT through freshly allocated device buffers; flags_host / bound_host optional.
static int crt_host(const char *name, const uint32_t *res, const uint32_t *primes, int P, int n_coeffs,
                    const uint32_t *bound_host, uint32_t *limbs_out, int limbs, uint32_t *flags_host) {
    CrtParams prm{};
    int rc = crt_params(primes, P, n_coeffs, limbs, &prm);
    if (rc) return rc;
    if (n_coeffs == 0) return CP_OK;
    if (!res || !limbs_out) return fail(CP_EINVAL, "NULL argument");
    uint32_t *r_d = nullptr, *l_d = nullptr, *b_d = nullptr, *f_d = nullptr;
    auto cleanup = [&]() {
        dev_free(r_d);
        dev_free(l_d);
        dev_free(b_d);
        dev_free(f_d);
    };
    if ((rc = dev_alloc((void **)&r_d, 4ull * P * n_coeffs)) || (rc = dev_alloc((void **)&l_d, 4ull * limbs * n_coeffs)) ||
        (flags_host && (rc = dev_alloc((void **)&f_d, 4ull * n_coeffs))) ||
        (flags_host && bound_host && (rc = dev_alloc((void **)&b_d, 4ull * n_coeffs)))) {
        cleanup();
        return rc;
    }
    cudaError_t e = cudaMemcpy(r_d, res, 4ull * P * n_coeffs, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && b_d) e = cudaMemcpy(b_d, bound_host, 4ull * n_coeffs, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        crt_kernel<<<(n_coeffs + 63) / 64, 64>>>(r_d, l_d, prm, b_d, f_d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(limbs_out, l_d, 4ull * limbs * n_coeffs, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && f_d) e = cudaMemcpy(flags_host, f_d, 4ull * n_coeffs, cudaMemcpyDeviceToHost);
    cleanup();
    if (e != cudaSuccess) return fail(CP_ECUDA, std::string(name) + ": " + cudaGetErrorString(e));
    return CP_OK;
}

// Count the flagged coefficients and turn them into CP_EPRIMES.
int cp::crt_outcome(const uint32_t *flags, int n_coeffs) {
    int nb = 0, nu = 0;
    for (int j = 0; j < n_coeffs; ++j) {
        nb += (flags[j] & 1u) ? 1 : 0;
        nu += (flags[j] & 2u) ? 1 : 0;
    }
    if (!nb && !nu) return CP_OK;
    return fail(CP_EPRIMES, "not enough primes: " + std::to_string(nb) + " coefficient(s) beyond the bound the "
                            "prime product covers, " + std::to_string(nu) + " not stable under dropping the "
                            "last prime");
}

extern "C" int cp_crt(const uint32_t *res, const uint32_t *primes, int P, int n_coeffs, uint32_t *limbs_out,
                      int limbs) {
    return crt_host("cp_crt", res, primes, P, n_coeffs, nullptr, limbs_out, limbs, nullptr);
}

extern "C" int cp_crt_checked(const uint32_t *res, const uint32_t *primes, int P, int n_coeffs,
                              const uint32_t *bound_bits, uint32_t *limbs_out, int limbs, uint32_t *flags_out) {
    std::vector<uint32_t> flags(n_coeffs > 0 ? n_coeffs : 1);
    int rc = crt_host("cp_crt_checked", res, primes, P, n_coeffs, bound_bits, limbs_out, limbs, flags.data());
    if (rc) return rc;
    if (flags_out)
        for (int j = 0; j < n_coeffs; ++j) flags_out[j] = flags[j];
    return crt_outcome(flags.data(), n_coeffs);
}

extern "C" int cp_whitney_bits(int lattice, int L, int N, int n_coeffs, uint32_t *bits_out) {
    if (lattice != CP_SQUARE && lattice != CP_TRIANGULAR) return fail(CP_EINVAL, "bad lattice");
    if (L < 1 || N < 1 || n_coeffs < 0 || (n_coeffs > 0 && !bits_out)) return fail(CP_EINVAL, "bad arguments");
    binomial_bits(rectangle_edges(lattice, L, N), n_coeffs, bits_out);
    return CP_OK;
}

// ------------------------------------------------------------------ primes

// Deterministic Miller-Rabin for n < 2^32 with bases 2, 7, 61.
__device__ bool is_prime_u32(uint32_t n) {
    if (n < 2) return false;
    const uint32_t small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 61};
    for (uint32_t q : small) {
        if (n == q) return true;
        if (n % q == 0) return false;
    }
    uint32_t d = n - 1;
    int r = 0;
    while ((d & 1) == 0) {
        d >>= 1;
        ++r;
    }
    const uint32_t bases[] = {2, 7, 61};
    for (uint32_t a : bases) {
        uint32_t x = powmod(a % n, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int k = 1; k < r; ++k) {
            x = mulmod(x, x, n);
            if (x == n - 1) {
                comp = false;
                break;
            }
        }
        if (comp) return false;
    }
    return true;
}

__global__ void next_prime_kernel(const uint64_t *draws, int n, uint32_t *out) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    uint64_t x = draws[k];
    uint32_t res = 0;
    // prime gaps below 2^32 are < 400: a bounded search
    for (int step = 0; step < 2000 && x < (1ull << 31); ++step, ++x)
        if (is_prime_u32((uint32_t)x)) {
            res = (uint32_t)x;
            break;
        }
    out[k] = res;
}

extern "C" int cp_select_primes(const uint64_t *draws, int n_draws, int n_primes, uint32_t *primes_out) {
    if (!draws || !primes_out || n_draws < 1 || n_primes < 1) return fail(CP_EINVAL, "bad arguments");
    uint64_t *d_d = nullptr;
    uint32_t *o_d = nullptr;
    int rc = dev_alloc((void **)&d_d, 8ull * n_draws);
    if (rc) return rc;
    if ((rc = dev_alloc((void **)&o_d, 4ull * n_draws))) {
        dev_free(d_d);
        return rc;
    }
    std::vector<uint32_t> cand(n_draws);
    cudaError_t e = cudaMemcpy(d_d, draws, 8ull * n_draws, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        next_prime_kernel<<<(n_draws + 127) / 128, 128>>>(d_d, n_draws, o_d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(cand.data(), o_d, 4ull * n_draws, cudaMemcpyDeviceToHost);
    dev_free(d_d);
    dev_free(o_d);
    if (e != cudaSuccess) return fail(CP_ECUDA, std::string("cp_select_primes: ") + cudaGetErrorString(e));
    int k = 0;
    for (int i = 0; i < n_draws && k < n_primes; ++i) {
        uint32_t p = cand[i];
        if (p == 0) continue;
        bool dup = false;
        for (int j = 0; j < k; ++j) dup = dup || primes_out[j] == p;
        if (!dup) primes_out[k++] = p;
    }
    if (k < n_primes) return fail(CP_EINVAL, "not enough distinct primes in the draws");
    return CP_OK;
}

// ------------------------------------------------------------------ diagnostics

namespace cp {
int debug_wait_timeout(long long cycles, cudaStream_t st);
int check_space(int kind, int m, int e, uint64_t *n_bad, uint64_t *size);
int enumerate_space(int kind, int m, int e, uint8_t *out_host, uint64_t max_states, uint64_t *size);
int debug_table(int lattice, int L, int paired, int which, int index, uint32_t *row_ptr_host, uint64_t max_rows,
                uint32_t *edges_host, uint64_t max_edges, uint64_t info[4]);
}  // namespace cp

extern "C" int cp_debug_table(int lattice, int L, int paired, int which, int index, uint32_t *row_ptr_host,
                              uint64_t max_rows, uint32_t *edges_host, uint64_t max_edges, uint64_t info[4]) {
    if ((lattice != CP_SQUARE && lattice != CP_TRIANGULAR) || L < 1 || L > CP_MAX_L || (which != 0 && which != 1))
        return fail(CP_EINVAL, "bad table");
    return debug_table(lattice, L, paired, which, index, row_ptr_host, max_rows, edges_host, max_edges, info);
}

extern "C" int cp_debug_check_space(int kind, int m, int e, uint64_t *n_bad, uint64_t *size) {
    if (m < 1 || m > CP_MAX_L || kind < 0 || kind > 2 || (kind == 1 && (e < 0 || e + 1 >= m)) ||
        (kind == 2 && m > CP_POTTS_MAX_L))
        return fail(CP_EINVAL, "bad space");
    return check_space(kind, m, e, n_bad, size);
}

extern "C" int cp_debug_wait_timeout(long long cycles) {
    if (cycles < 0 || cycles > (1ll << 33)) return fail(CP_EINVAL, "cycles must be in [0, 2^33]");
    return debug_wait_timeout(cycles, 0);
}

extern "C" int cp_debug_enumerate_space(int kind, int m, int e, uint8_t *out_host, uint64_t max_states,
                                        uint64_t *size) {
    if (m < 1 || m > CP_MAX_L || kind < 0 || kind > 2 || (kind == 1 && (e < 0 || e + 1 >= m)) ||
        (kind == 2 && m > CP_POTTS_MAX_L))
        return fail(CP_EINVAL, "bad space");
    return enumerate_space(kind, m, e, out_host, max_states, size);
}

// ------------------------------------------------------------------ CRT without allocation
//
// cp_crt allocates two device buffers on every call.  Some callers cannot do
// that: a process whose device memory is entirely handed to another allocator
// (a framework's caching allocator, a fixed arena reserved at start-up), or a
// service that forbids new device allocations once it is serving.
// cp_crt_static runs the same kernel with its residues and limbs staged in
// this fixed device array instead.  The array belongs to this file's device
// module: CUDA loads a module on a device (and with it the array's 8 MiB) when
// the module is first used there, which the library's set-up calls do (see
// crt_static_touch); it is then held until the process exits.

static __device__ __align__(256) uint8_t g_crt_scratch[CP_CRT_STATIC_BYTES];

// Device address of the array in the current device's context.  Looked up on
// every call (a cheap query next to the two synchronous copies of a call), so
// no address outlives the context it was taken in.
static int crt_static_scratch(uint8_t **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_crt_scratch);
    if (e != cudaSuccess || !p)
        return fail(CP_ECUDA, std::string("cudaGetSymbolAddress(g_crt_scratch): ") + cudaGetErrorString(e));
    *out = (uint8_t *)p;
    return CP_OK;
}

namespace cp {
// Load this module (and the static array) on the current device; the strip,
// sweep and server set-up calls make it, so that a caller who creates any of
// them before handing the rest of the device memory to another allocator has
// the array in place.
int crt_static_touch() {
    uint8_t *p = nullptr;
    return crt_static_scratch(&p);
}
}  // namespace cp

extern "C" int cp_crt_static(const uint32_t *res, const uint32_t *primes, int P, int n_coeffs, uint32_t *limbs_out,
                             int limbs) {
    CrtParams prm{};
    int rc = crt_params(primes, P, n_coeffs, limbs, &prm);
    if (rc) return rc;
    if (n_coeffs == 0) return CP_OK;
    if (!res || !limbs_out) return fail(CP_EINVAL, "NULL argument");
    const size_t res_bytes = 4ull * P * n_coeffs;
    const size_t res_span = (res_bytes + 255) & ~(size_t)255;
    const size_t limb_bytes = 4ull * limbs * n_coeffs;
    if (res_span + limb_bytes > CP_CRT_STATIC_BYTES)
        return fail(CP_EINVAL, "cp_crt_static: residues (" + std::to_string(res_bytes) + " bytes) plus limbs (" +
                                   std::to_string(limb_bytes) + " bytes) exceed CP_CRT_STATIC_BYTES (" +
                                   std::to_string((size_t)CP_CRT_STATIC_BYTES) + ")");
    uint8_t *base = nullptr;
    if ((rc = crt_static_scratch(&base))) return rc;
    uint32_t *r_d = reinterpret_cast<uint32_t *>(base);
    uint32_t *l_d = reinterpret_cast<uint32_t *>(base + res_span);
    // the kernel reads only the residues copied here and writes every limb, so no
    // part of the array has to be cleared between calls
    cudaError_t e = cudaMemcpy(r_d, res, res_bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        crt_kernel<<<(n_coeffs + 63) / 64, 64>>>(r_d, l_d, prm, nullptr, nullptr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(limbs_out, l_d, limb_bytes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(CP_ECUDA, std::string("cp_crt_static: ") + cudaGetErrorString(e));
    return CP_OK;
}
