// Internal declarations shared by the translation units of libcp_gb300.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>
#include <string>
#include <vector>

#include "cp_tm.h"

namespace cp {

// ------------------------------------------------------------------ errors
void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
// Distinct primes in [2, 2^31), 1..CP_MAX_PRIMES of them (trial division on the host).
int check_primes(const uint32_t *primes, int n);

#define CP_CUDA_TRY(expr)                                                                \
    do {                                                                                 \
        cudaError_t _e = (expr);                                                         \
        if (_e != cudaSuccess)                                                           \
            return ::cp::fail(CP_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
    } while (0)

// ------------------------------------------------------------------ state spaces
// Point counts go up to CP_MAXN in the rank tables (contracted spaces use L-1).
constexpr int kMaxN = 24;
constexpr int kTblStride = kMaxN + 1;

// cnt[n] = number of NCNNN partitions of n points (cnt[0] = 1, cnt[n] = M_{n-1});
// off[n*kTblStride + k] = rank of the first n-point partition whose first point
// has its smallest partner at relative position 2+k (eq. (M_recurs)).
// cntc[n] = Catalan C_n (non-crossing partitions of n points), offc[n*kTblStride + k]
// = rank of the first n-point non-crossing partition whose first point has its
// smallest partner at relative position 1+k.
struct RankTables {
    uint64_t cnt[kTblStride];
    uint64_t off[kTblStride * kTblStride];
    uint64_t cntc[kTblStride];
    uint64_t offc[kTblStride * kTblStride];
};

// A state space of one per-site factor.
//  SPACE_B: NCNNN partitions in the paper's order (first `size` ranks).
//  SPACE_X: partitions NCNNN except that e ~ e+1 is allowed (square lattice,
//           Sec. 3.4).  Ordered by interleaving: the NCNNN partitions in B
//           order, each NCNNN partition t in which e is alone and e-1 !~ e+1
//           immediately followed by J_{e,e+1} t.  prefix[b] = number of such t
//           with B-rank < b, so rank(t) = b + prefix[b] and rank(J t) = that + 1.
//  SPACE_C: all non-crossing partitions (the any-v Potts model, Sec. 3.2), in
//           the order: first point alone first, then by its smallest partner.
enum SpaceKind : int32_t { SPACE_B = 0, SPACE_X = 1, SPACE_C = 2 };
struct Space {
    int32_t kind;
    int32_t m;      // number of sites
    int32_t e;      // excepted pair (SPACE_X)
    int32_t pad;
    uint64_t size;  // number of ranks used
    const uint32_t *prefix;  // SPACE_X: [M_{m-1} + 1] on the device
};

// Kind of per-site factor.
enum OpKind : int32_t {
    OP_SQUARE = 0, OP_TRIANGULAR = 1, OP_LAST = 2, OP_IDENTITY = 3,  // chromatic (v = -1, projected)
    OP_POTTS_SQUARE = 4, OP_POTTS_TRIANGULAR = 5, OP_POTTS_LAST = 6  // any v, no projectors
};

struct OpDesc {
    int32_t kind;
    int32_t m;
    int32_t i;       // 0-based site
    int32_t max_terms;
    Space in, out;
    int32_t v;         // Potts coupling (OP_POTTS_*)
    int32_t src_bits;  // edge format of the table
    int32_t fused;     // 1: two-site table, factor (kind_b, i_b) applied after (kind, i)
    int32_t kind_b;
    int32_t i_b;
    int32_t pad2;
};

// Packed CSR edge: src (src_bits) | shift << src_bits (2 bits) | coef << (src_bits + 2)
// (two's complement in the remaining bits).  Chromatic tables: 27 / 2 / 3 bits
// (coefficients +1, -1, -2, -3).  Potts tables take as few source bits as the
// space needs (at least 16), leaving 30 - src_bits bits for the coefficient.
constexpr uint32_t kSrcBits = 27;
constexpr uint32_t kSrcMask = (1u << kSrcBits) - 1u;
constexpr uint32_t kPottsMinSrcBits = 16;
inline int potts_src_bits(uint64_t n_states) {
    int b = (int)kPottsMinSrcBits;
    while (b < (int)kSrcBits && (1ull << b) - 1 < n_states) ++b;
    return b;
}

// CSR-by-destination table of one per-site factor, on the device.
struct SiteTable {
    OpDesc op;
    uint64_t n_src = 0, n_dst = 0, nnz = 0;
    uint64_t n_site_out = 0;  // output states of the per-site factors it stands for (n_dst, or mid + n_dst)
    uint32_t *row_ptr = nullptr;  // [n_dst + 1]
    uint32_t *edges = nullptr;    // [nnz]
    uint32_t *block_order = nullptr;  // row blocks by smallest source (GatherTask::block_order), or null
    uint32_t max_coef_sum = 0;        // largest sum of |coefficient| into one destination (an upper bound)
    uint32_t max_abs_coef = 0;        // largest |coefficient|
};

// All tables of one (lattice, L) on one device; shared between strips.
struct TableSet {
    int device = 0, lattice = 0, L = 0, potts = 0, v = -1, src_bits = (int)kSrcBits, paired = 0;
    uint64_t S_b = 0, S_max = 0;
    // T_1..T_L and T_1^last..T_{L-1}^last (identity for L = 1), one table per
    // factor, or (paired) one two-site table per consecutive pair of factors
    // (T_2 T_1, T_4 T_3, ...; an odd one out stays single)
    std::vector<SiteTable> row;
    std::vector<SiteTable> last;
    std::vector<uint32_t *> x_prefix;  // square lattice: prefix table of X_e, e = 0..L-2
    size_t bytes = 0;
    ~TableSet();
};

// Rank tables on the current device (built once per device by a kernel).
int device_rank_tables(const RankTables **out_dev, RankTables *host_copy);

// Prefix table of the interleaved space X_e on m sites (device, [M_{m-1} + 1]).
int build_x_prefix(int m, int e, cudaStream_t st, uint32_t **out);

// Build or fetch from the cache the tables of (lattice, L) on the current device
// (chromatic polynomial: the projected factorisation of Sec. 3.2-3.3), paired
// or not according to factor_pairing() and the row size.
// row_bytes = bytes of one state's row, (D+1) * n_primes * 4, of the caller's vectors.
int get_tables(int lattice, int L, size_t row_bytes, cudaStream_t stream, std::shared_ptr<TableSet> *out);
// Library-wide choice for tables built from now on: 0 = one table per factor, 1 = two-site
// square-lattice tables for rows of at least kPairRowBytes (default), 2 = every square table.
constexpr size_t kPairRowBytes = 3072;
int factor_pairing();
int set_factor_pairing(int mode);
// Tables of the any-v Potts transfer matrix T_i = V_i H_{i,i+1} (square) or
// V_i H_{i-1,i} H_{i,i+1} (triangular) on non-crossing partitions.
int get_potts_tables(int lattice, int L, int v, cudaStream_t stream, std::shared_ptr<TableSet> *out);

// ------------------------------------------------------------------ gather
// One per-site factor application: out[dst] = sum_e coef_e * w^{shift_e} in[src_e]  (mod p)
struct GatherTask {
    const uint32_t *in;
    uint32_t *out;
    const uint32_t *row_ptr;
    const uint32_t *edges;
    const uint32_t *primes;   // n_primes words, device
    uint32_t rows;            // destination rows of this task
    uint32_t C;               // chunks per row (16-byte chunks if vec4, else words)
    uint32_t cpd;             // chunks per degree (= n_primes / VEC)
    uint32_t vec4;            // 1: 16-byte chunks, 0: 4-byte chunks
    uint32_t block_begin;     // first block of this task in the launch
    uint32_t magic_cpd;       // x / cpd = umulhi(x, magic_cpd) for x * cpd < 2^32 (0: cpd == 1)
    uint32_t n_primes;
    uint32_t c0;              // first chunk of the rows handled by this task
    uint32_t cw;              // chunks handled (a column range [c0, c0 + cw) of every row)
    uint32_t src_bits;        // edge format of the table
    uint32_t partial;         // 1: the output feeds further gathers only (words may be left in [-p, p))
    uint32_t small_coefs;     // 1: |coefficient| <= 127 and their sum into any destination < 2^15 (TMA kernel)
    // TMA kernel: the order in which its blocks visit the row blocks, for 16,
    // 32, 64 and 128 rows per block one after another (block_order_offset),
    // or null for row-block order
    const uint32_t *block_order;
};

// Start of the order for `rpb` rows per block in a table of `rows` rows.
__host__ __device__ inline uint32_t block_order_offset(uint32_t rows, uint32_t rpb) {
    uint32_t off = 0;
    for (uint32_t l = 16; l < rpb; l *= 2) off += (rows + l - 1) / l;
    return off;
}

constexpr int kGatherThreads = 256;  // 8 warps; one warp per destination row at a time
constexpr int kGatherItems = 4;      // default rows per warp (the tile: 8 * rows per block)

// Append the task(s) of one per-site factor: rows of 16-byte chunks wider than
// 256 chunks are split into column tasks of at most 256 chunks each.
// partial: the output vector is read by further gathers only, so the TMA kernel
// may store signed representatives in [-p, p) (every gather reads its input
// words as signed 32-bit values).
void append_gather_tasks(std::vector<GatherTask> *tasks, const SiteTable &tab, const uint32_t *in,
                         uint32_t *out, const uint32_t *primes_dev, int D1, int P, bool partial = false);
// Gather tile (low 12 bits): 1, 2, 4, 8 = register kernel with that many rows
// per warp (8 warps per block); 16, 32, 64, 128 = TMA kernel with that many rows
// per block.  For TMA tiles, bits 12..19 = ring size in KB (0: default) and
// bits 20..23 = edges per stage, 1, 2, 4 or 8 (0: picked from the row size),
// bits 24..27 = 16-byte chunks per consumer thread, 1, 2 or 4 (0: 2 for rows
// wider than 3 KB, else 1), bits 28..29 = consumer block shape, 1 = wide
// (8 / chunks-per-thread consumer warps), 2 = narrow (5 consumer warps, one
// chunk per thread, rows of at most 160 chunks), 0 = narrow for batches whose
// rows all have 129..160 chunks at one chunk per thread, else wide.  A batch
// whose rows are not all 16-byte chunked uses the register kernel.
constexpr int kTmaRingKbDefault = 48;
constexpr int kTileWide = 1 << 28;
constexpr int kTileNarrow = 2 << 28;
constexpr int kTmaNarrowWarps = 5;  // consumer warps of a narrow block
inline int make_tile(int rows, int ring_kb, int edges = 0, int cpt = 0) {
    return rows | (ring_kb << 12) | (edges << 20) | (cpt << 24);
}
inline int tile_edges(int tile) { return (tile >> 20) & 15; }
inline int tile_cpt(int tile) { int c = (tile >> 24) & 15; return c ? c : 1; }
inline int tile_ring_kb(int tile) { int r = (tile >> 12) & 0xFF; return r ? r : kTmaRingKbDefault; }
inline int tile_shape(int tile) { return (tile >> 28) & 3; }
// Blocks per SM the TMA kernel's launch bounds aim at (its registers), and the
// shared-memory ring that fills the SM at that occupancy; W = consumer warps
// (0: the wide block, 8 / CPT).
__host__ __device__ constexpr int tma_min_blocks(int E, int CPT, int W = 0) {
    return W == kTmaNarrowWarps ? 4
                                : (CPT == 1 ? (E >= 2 ? 3 : 4) : (CPT == 2 ? 4 : (E >= 4 ? 4 : 5)));
}
__host__ __device__ constexpr int tma_ring_kb_for(int E, int CPT, int W = 0) {
    return W == kTmaNarrowWarps ? 52
                                : (tma_min_blocks(E, CPT) <= 3 ? 64 : (tma_min_blocks(E, CPT) == 4 ? 48 : 40));
}
bool tile_is_tma(int items);
bool tma_usable(const GatherTask &t);
// Blocks of one task and of a whole launch (fills block_begin; returns the grid size).
uint32_t task_blocks(const GatherTask &t, int items);
uint32_t assign_blocks(std::vector<GatherTask> &tasks, int items);
// Effective tile for a batch (falls back from TMA to the register kernel when needed).
int effective_tile(const std::vector<GatherTask> &tasks, int items);
// The TMA kernel accumulates coef * x as two 16 x 8-bit dot products into 32-bit
// halves (gather_tma.cu), exact while |coef| <= kTmaMaxCoef and the sum of
// |coef| into any destination stays below kTmaMaxCoefSum; other tables use the
// register kernel.
constexpr uint32_t kTmaMaxCoef = 127;
constexpr uint32_t kTmaMaxCoefSum = 1u << 15;
// Rows per block of the default TMA tile for a launch of these tasks (16 or 32).
int default_rows(const std::vector<GatherTask> &tasks);
// Launch a batch of tasks (tasks_dev = device copy, block_begin assigned for `items`).
int launch_gather(const GatherTask *tasks_dev, int n_tasks, uint32_t total_blocks, int items, cudaStream_t st);
// Set the kernels' shared-memory attributes (call outside stream capture).
int prepare_gather_kernels();
// Device error word set by bounded waits in kernels; check_device_error syncs
// `st`, returns CP_ETIMEOUT (and clears the word) if it was set.
int *device_error_flag();
int check_device_error(cudaStream_t st);

// Extract the e0 row laid out [D1][P] into [P][D1].
int launch_transpose_row(const uint32_t *row, uint32_t *out, int D1, int P, cudaStream_t st);

// ------------------------------------------------------------------ CRT (crt.cu)
// Device CRT of residues [P][n_coeffs] into limbs [n_coeffs][limbs]; with
// flags_dev, per-coefficient flags (bit 0: bound_dev[j] + 2 > bit length of the
// prime product; bit 1: the first P-1 primes give another value).
int launch_crt(const uint32_t *res_dev, const uint32_t *primes_host, int P, int n_coeffs, uint32_t *limbs_dev,
               int limbs, const uint32_t *bound_dev, uint32_t *flags_dev, cudaStream_t st);
int primes_product_bits(const uint32_t *primes, int P);
// Bit lengths of C(n_edges, j), j < n_coeffs (Whitney's bound |c_j| <= C(|E|, j)).
void binomial_bits(uint64_t n_edges, int n_coeffs, uint32_t *bits_out);
uint64_t rectangle_edges(int lattice, int L, int N);
// CP_OK if no flag is set, else CP_EPRIMES with a message counting them.
int crt_outcome(const uint32_t *flags, int n_coeffs);
// Load the CRT module (and the static array of cp_crt_static) on the current device.
int crt_static_touch();

// Device allocation helpers (library-owned memory).
int dev_alloc(void **p, size_t bytes);
void dev_free(void *p);

}  // namespace cp
