/*
 * cp_tm.h -- C ABI of the GB300 chromatic-polynomial transfer-matrix library.
 *
 * Computes P~_G(q) = q^{-|V|} P_G(q) (a polynomial in w = 1/q with constant
 * term 1, eq. (Z_modified), Sec. 3.5) for L x N rectangles of the square and
 * triangular lattices with free boundaries, as residues modulo 31-bit primes,
 * with the sparse per-site transfer matrix of Jacobsen, arXiv:1005.3609:
 *   P~ = <e_0| T_last T^{N-1} |e_0>,                       eq. (Z_from_T)
 *   T = T_L ... T_1, per-site factors eqs. (T_sq_proj) / Sec. 3.3,
 *   T_last = T_L^last ... T_1^last,                         eqs. (T_last), (T_last_i)
 * acting on vectors indexed by the rank of non-crossing non-nearest-neighbour
 * (NCNNN) partitions of the L top-row sites (Sec. 3.4).
 *
 * Conventions for every entry point:
 *  - Return CP_OK (0) or a negative status; nothing throws across the ABI.
 *    The thread-local message of the last failure is cp_last_error().
 *  - Pointers named *_host are host memory owned by the caller; pointers named
 *    *_dev are device memory (cudaMalloc/torch) owned by the caller.
 *  - Library objects (cp_strip, cp_sweep, cp_server) own their device memory
 *    until the matching destroy call.
 *  - cuda_stream is a cudaStream_t passed as void*; NULL = legacy default stream.
 *  - Primes must be distinct primes in [2, 2^31); residues are uint32 < p.
 *  - Residue arrays of one polynomial are laid out [n_primes][D+1]:
 *    out[k*(D+1) + j] = coefficient of w^j modulo primes[k].
 */
#ifndef CP_TM_H
#define CP_TM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { CP_SQUARE = 0, CP_TRIANGULAR = 1 };

enum {
    CP_OK = 0,
    CP_EINVAL = -1,   /* bad argument                                   */
    CP_ENOMEM = -2,   /* device or host allocation failed / over budget */
    CP_ECUDA = -3,    /* a CUDA call failed                             */
    CP_ETIMEOUT = -4, /* a bounded device wait ran out                  */
    CP_ESTATE = -5,   /* internal consistency check failed              */
    CP_EPRIMES = -6   /* too few primes for an exact integer result     */
};

#define CP_MAX_L 20       /* widest strip compiled in (the paper's m_max = 20, Sec. 4.2) */
#define CP_MAX_PRIMES 32
#define CP_POTTS_MAX_L 16 /* widest any-v Potts strip (Catalan(16) = 35,357,670 states) */
#define CP_POTTS_MAX_V 16 /* |v| bound of the Potts strip (see cp_create_strip_potts) */

typedef struct cp_strip cp_strip;

/*
 * cp_create_strip -- a strip of width L, height 1, state vector = e_0.
 * Builds (or reuses from the per-device cache) the rank tables and the CSR
 * tables of every per-site factor T_i and T_i^last on the GPU, and allocates
 * the two state vectors [S][D+1][n_primes] (S = M_{L-1} + M_{L-2} on the
 * square lattice, M_{L-1} on the triangular one; Sec. 3.2-3.3).
 *   lattice    CP_SQUARE or CP_TRIANGULAR
 *   L          1..CP_MAX_L sites per row (strip width m of the paper)
 *   primes_host, n_primes   1..CP_MAX_PRIMES distinct primes < 2^31 (copied)
 *   max_degree D >= 0 keeps w^0..w^D (truncation, Sec. 3.5); -1 = full degree
 *              L*max_rows - 1
 *   max_rows   height limit (>= 1); advancing beyond it is CP_EINVAL
 * Errors: CP_EINVAL (bad lattice/L/primes/D), CP_ENOMEM, CP_ECUDA, CP_ESTATE.
 */
int cp_create_strip(int lattice, int L, const uint32_t *primes_host, int n_primes,
                    int max_degree, int max_rows, void *cuda_stream, cp_strip **out);

/*
 * cp_create_strip_potts -- the same strip for the Potts partition function at
 * any integer v (Sec. 3.1-3.2, the construction T = (prod_i V_i)(prod_i H_{i,i+1})
 * before the chromatic specialisation): Z~(w) = q^{-|V|} Z(q, v) as a polynomial
 * in w = 1/q, Z(q, v) = sum over edge subsets A of q^{k(A)} v^{|A|}, with
 *   H_{i,i+1} = 1 + v J_{i,i+1},   V_i = v w + D_i,
 * on all non-crossing partitions of the L sites (Catalan(L) states, no
 * projector), triangular rectangles with the diagonals of Sec. 3.3.  At v = -1
 * the residues equal those of cp_create_strip.  The strip is driven by the same
 * calls (cp_advance_rows, cp_read_coeffs, cp_strip_info with n_states[0] =
 * n_states[1] = Catalan(L), cp_strip_reset, cp_destroy).
 *   v          integer coupling, |v| <= CP_POTTS_MAX_V; residues are taken mod
 *              each prime, so v stands for its residue class
 *   L          1..CP_POTTS_MAX_L
 *   other arguments as cp_create_strip
 * The transition coefficients (products of v and 1 + v) are packed beside a
 * source index that needs ceil(log2 Catalan(L)) bits; the 30 - that many bits
 * left hold the coefficient.  A v whose coefficients do not fit at this width
 * is CP_EINVAL with a message saying so (wide strips take smaller |v|).
 * Errors: CP_EINVAL (bad lattice/L/v/primes/D, coefficient too wide),
 * CP_ENOMEM, CP_ECUDA, CP_ESTATE.
 */
int cp_create_strip_potts(int lattice, int L, int v, const uint32_t *primes_host, int n_primes,
                          int max_degree, int max_rows, void *cuda_stream, cp_strip **out);

/*
 * cp_advance_rows -- apply T = T_L ... T_1 n_rows times (eq. (T_sq_decomp));
 * height += n_rows.  Asynchronous on the strip's stream (one gather launch per
 * table: per site, or per pair of sites with two-site tables).
 * Errors: CP_EINVAL (height would exceed max_rows), CP_ECUDA.
 */
int cp_advance_rows(cp_strip *s, int n_rows);

/*
 * cp_read_coeffs -- P~ of the L x height rectangle: applies T_last to a copy
 * of the state vector and extracts the e_0 coefficient (eqs. (T_last_i),
 * (Z_from_T)).  Writes out_host[n_primes][D+1] (out_len >= n_primes*(D+1)
 * words) and *height_out; synchronises the strip's stream.
 */
int cp_read_coeffs(cp_strip *s, uint32_t *out_host, size_t out_len, int *height_out);

/* As cp_read_coeffs, into device memory out_dev[n_primes][D+1], asynchronous on
 * the strip's stream (no host synchronisation). */
int cp_read_coeffs_device(cp_strip *s, uint32_t *out_dev, size_t out_len);

/* Strip geometry: n_states[0] = NCNNN states S_b, n_states[1] = largest
 * intermediate space, *degree = D, *height = current height. */
int cp_strip_info(const cp_strip *s, uint64_t n_states[2], int *degree, int *height);

/* Work of the strip's factors, for throughput and roofline figures:
 * work[0] = updates of one row advance (output words of T_1 .. T_L: sum of
 * S_out (D+1) n_primes over the per-site factors), work[1] = the bytes its
 * launched tables need (each reads its input vector and writes its output
 * vector once, 4 (S_in + S_out)(D+1) n_primes, plus its CSR table,
 * 4 (S_out + 1 + nnz); a two-site table skips the intermediate vector),
 * work[2], work[3] = the same for one read-out (T_1^last .. T_{L-1}^last),
 * work[4], work[5] = the bytes of the row and of the read-out done one factor
 * at a time (intermediate vectors included).  No GPU work. */
int cp_strip_work(const cp_strip *s, uint64_t work[6]);

/* Gather tile of the strip's launches, encoded as cp_sweep_create's tile
 * (0 = the default: TMA kernel, 32 rows per block -- 16 where 32-row blocks
 * would give a launch fewer than eight waves of resident blocks -- stages,
 * chunks per thread and ring picked from the row width).  A tuning knob: results are identical
 * for every tile.  Synchronises the strip's stream.  CP_EINVAL on a bad tile. */
int cp_strip_set_tile(cp_strip *s, int tile);

/* Restart the strip at height 1 with the state vector e_0 (keeps its tables
 * and buffers).  Asynchronous on the strip's stream. */
int cp_strip_reset(cp_strip *s);

void cp_destroy(cp_strip *s);

/*
 * cp_set_factor_pairing -- how the chromatic tables built from
 * now on are laid out (strips, sweeps and server jobs created afterwards;
 * tables already built stay cached under their own layout).  A two-site table
 * is the product of a consecutive pair of per-site factors, T_2 T_1, T_4 T_3,
 * ... of the row and of the read-out chain (an odd one out stays single): a
 * row of L sites takes ceil(L/2) gather launches and the intermediate vector
 * of each pair is never written -- the same matrix product as the
 * factorisation of Sec. 3.2 with half the vector traffic but as many edge
 * copies, which pays only when a state's row, (D+1) n_primes words, is a few
 * KB long.  mode 1 (the default): two-site tables for square-lattice rows of
 * at least 3 KB; mode 2: for every square-lattice strip; mode 3: for every
 * strip of both lattices; mode 0: one table per factor, as in the paper.
 * Results are identical in every mode.  Returns the previous mode.  Not thread-safe
 * against concurrent strip creation.
 */
int cp_set_factor_pairing(int mode);

/*
 * cp_crt -- Chinese remaindering (Sec. 3.5): for each of n_coeffs
 * coefficients, residues_host[k*n_coeffs + j] modulo primes_host[k] ->
 * the integer in (-prod/2, prod/2], written as limbs_per_coeff little-endian
 * 32-bit limbs in two's complement: limbs_host[j*limbs_per_coeff + l].
 * Runs on the GPU (Garner's mixed radix, one thread per coefficient).  It
 * returns whatever the given primes determine: an integer of magnitude
 * prod/2 or more comes back reduced; cp_crt_checked says when that may be so.
 * Errors: CP_EINVAL if limbs_per_coeff * 32 is below the bit length of
 * prod(primes) plus 1 (computed exactly), or bad primes.
 */
int cp_crt(const uint32_t *residues_host, const uint32_t *primes_host, int n_primes,
           int n_coeffs, uint32_t *limbs_host, int limbs_per_coeff);

/*
 * cp_crt_checked -- cp_crt plus the two sufficiency checks of the
 * reconstruction (Sec. 3.5: primes are added until the result stops changing).
 * Per coefficient j, flags_host[j] (optional, may be NULL) gets
 *   bit 0: bound_bits_host is given and bound_bits_host[j] + 2 exceeds the bit
 *          length of prod(primes), i.e. a coefficient with |c_j| < 2^bound_bits
 *          is not guaranteed to lie in the recovered range (-prod/2, prod/2);
 *   bit 1: the value recombined from the first n_primes - 1 primes differs
 *          from the one from all n_primes (always set for n_primes = 1).
 * bound_bits_host may be NULL (stabilisation check only); for chromatic
 * polynomials cp_whitney_bits gives a valid bound.  The limbs are written in
 * any case; the return is CP_EPRIMES ("not enough primes", with the counts in
 * cp_last_error()) if any flag is set, else CP_OK.  Other errors as cp_crt.
 */
int cp_crt_checked(const uint32_t *residues_host, const uint32_t *primes_host, int n_primes, int n_coeffs,
                   const uint32_t *bound_bits_host, uint32_t *limbs_host, int limbs_per_coeff,
                   uint32_t *flags_host);

/*
 * cp_whitney_bits -- bits_host[j] = bit length of C(|E|, j), j < n_coeffs, for
 * the L x N rectangle of the lattice (|E| = L(N-1) + N(L-1), plus (L-1)(N-1)
 * diagonals on the triangular lattice).  By Whitney's broken-circuit theorem
 * the coefficient of q^{|V|-j} in P_G(q), which is c_j of P~ (eq.
 * (Z_modified)), satisfies |c_j| <= C(|E|, j), so these are bounds for
 * cp_crt_checked.  Exact integer arithmetic on the host; no GPU work.
 */
int cp_whitney_bits(int lattice, int L, int N, int n_coeffs, uint32_t *bits_host);

/*
 * cp_read_integers -- the exact integer coefficients c_0..c_D of the strip's
 * P~ (L x height): the read-out of cp_read_coeffs, then the CRT over the
 * strip's primes on the GPU with both checks of cp_crt_checked (chromatic
 * strips: Whitney's bound for L x height and stabilisation; Potts strips:
 * stabilisation only).  Writes limbs_host[j*limbs_per_coeff + l] (limbs_len >=
 * (D+1)*limbs_per_coeff), flags_host[0..D] if not NULL, *height_out if not
 * NULL; synchronises the strip's stream.  Returns CP_EPRIMES when the strip's
 * primes are too few for an exact result (the limbs are still written).
 * Errors: CP_EINVAL (sizes, limbs_per_coeff too small for the prime product),
 * CP_ENOMEM, CP_ECUDA, CP_ETIMEOUT.
 */
int cp_read_integers(cp_strip *s, uint32_t *limbs_host, size_t limbs_len, int limbs_per_coeff,
                     uint32_t *flags_host, int *height_out);

/* Device-memory variant of cp_crt (asynchronous on cuda_stream). */
int cp_crt_device(const uint32_t *residues_dev, const uint32_t *primes_host, int n_primes,
                  int n_coeffs, uint32_t *limbs_dev, int limbs_per_coeff, void *cuda_stream);

/*
 * cp_crt_static -- cp_crt without any device allocation.  The paper has no
 * counterpart: this is a service of the library.  cp_crt allocates device
 * buffers on every call; callers that cannot allocate device memory (their
 * device memory is entirely owned by another allocator, or their service
 * forbids new allocations once it runs) use this entry point instead.  Same
 * arguments, result and errors as cp_crt.  The residues and limbs are staged in
 * one fixed device array of CP_CRT_STATIC_BYTES bytes (residues rounded up to
 * 256 bytes, then limbs); a call needing more returns CP_EINVAL with the sizes
 * in cp_last_error().  The array lives in the library's CRT device module.
 * CUDA loads a module onto a device lazily, when the module is first used
 * there, and that is when the array's 8 MiB are taken on that device (held
 * until the process exits): the first cp_crt_static call on the device, or any
 * earlier cp_select_primes, cp_crt*, cp_create_strip*, cp_sweep_create or
 * cp_server_create call there.  A caller whose allocator is about to take the
 * rest of the device memory makes one of these calls on each device first.
 * Each call looks up the array's device address (cudaGetSymbolAddress) with
 * the calling thread's current device, so the first call on a device should
 * come before any stream capture.  Synchronous (legacy default stream).  All
 * calls share the array and it keeps the last call's contents (every limb is
 * rewritten, nothing needs clearing), so calls that overlap on the GPU -- from
 * several host threads at once -- race; serialise them.
 */
#define CP_CRT_STATIC_BYTES (8u << 20)
int cp_crt_static(const uint32_t *residues_host, const uint32_t *primes_host, int n_primes,
                  int n_coeffs, uint32_t *limbs_host, int limbs_per_coeff);

/*
 * cp_select_primes -- the prime set (Sec. 3.5 leaves the choice open): each
 * draw in [2^30, 2^31) is mapped on the GPU to the smallest prime >= draw
 * (deterministic Miller-Rabin, bases 2, 7, 61); repeats and results >= 2^31
 * are skipped; the first n_primes are written to primes_host.
 * Errors: CP_EINVAL if the draws yield fewer than n_primes primes.
 */
int cp_select_primes(const uint64_t *draws_host, int n_draws, int n_primes, uint32_t *primes_host);

/* ---------------------------------------------------------------- batched sweep
 * The finite-lattice sweep of Sec. 4.1-4.3: every rectangle r x s with r <= s
 * and k-3 <= r+s <= k (the rectangles of B(k) with a non-zero weight,
 * eqs. (fb)-(fc)), on n_primes primes, truncated to the series order: square
 * lattice 2k-3 terms in z (2k-2 for odd k, with the mu_{2m} z^{4m-1} terms of
 * Sec. 4.2 added to f_b and f_s), triangular lattice k terms in x (Sec. 4.3).
 * One strip per width (and per prime group) is advanced to its largest band
 * height and read out at each band height; all strips advance together, one
 * batched launch per site step, and the whole sweep plus the series kernel is
 * one CUDA graph.
 */
typedef struct cp_sweep cp_sweep;

/* tile: 0 = autotune; 1, 2, 4, 8 = register gather kernel, rows per warp;
 *       16, 32, 64, 128 = TMA gather kernel, rows per block, optionally plus
 *       (ring KB << 12) with ring KB in 16..192 (shared-memory ring per block,
 *       0 = what fills the SM at the kernel's occupancy; raised to hold two
 *       stages), (edges per stage << 20) with 1, 2, 4 or 8 (0 = about 20 KB
 *       of source rows per stage, at most 32 / row groups; 4 in narrow blocks), (16-byte chunks
 *       per consumer thread << 24) with 1, 2 or 4 (0 = 2 for rows wider than
 *       3 KB, else 1) and (block shape << 28) with 1 = wide (8 / chunks-per-
 *       thread consumer warps) or 2 = narrow (5 consumer warps; one chunk per
 *       thread, rows of at most 160 chunks) (0 = narrow where every row of a
 *       launch has 129..160 chunks at one chunk per thread, else wide);
 * prime_groups: number of strips per width, dividing n_primes, or 0 = autotune.
 * cuda_stream must be a non-default stream (the program is graph-captured on it).
 * Errors: CP_EINVAL (k < 4, k/2 > CP_MAX_L, series longer than 128 terms, bad
 * primes/tile/groups, NULL stream), CP_ENOMEM, CP_ECUDA, CP_ESTATE. */
int cp_sweep_create(int lattice, int k, const uint32_t *primes_host, int n_primes, int tile, int prime_groups,
                    void *cuda_stream, cp_sweep **out);

/* Launch the whole sweep (one graph launch), asynchronous on the sweep's stream. */
int cp_sweep_run(cp_sweep *sw);

/* Wait for the sweep's stream; CP_ESTATE if a P~ had a constant term != 1. */
int cp_sweep_sync(cp_sweep *sw);

/* Geometry and algorithmic work of one run: output words written by the
 * per-site factors (updates) and bytes = 4 (S_in + S_out)(D+1) P per factor
 * plus its CSR index; launches = batched gather launches + 1 series kernel. */
int cp_sweep_info(const cp_sweep *sw, int *n_rects, int *n_terms, int *tile, int *prime_groups,
                  uint64_t *updates_per_run, uint64_t *bytes_per_run, int *launches_per_run);

/* Work of one run in both accountings: work[0] = updates (output words of
 * every per-site factor, as in cp_sweep_info), work[1] = bytes the launched
 * tables need (input + output vector + CSR of each table, two-site tables
 * included: as bytes_per_run), work[2] = bytes of the same work done one
 * factor at a time (4 (S_in + S_out)(D+1) P for every per-site factor, the
 * intermediate vectors of two-site tables included, plus the tables' CSR). */
int cp_sweep_work(const cp_sweep *sw, uint64_t work[3]);

/* The rectangles, rs_host[2j] = r, rs_host[2j+1] = s. */
int cp_sweep_rects(const cp_sweep *sw, int *rs_host, int max_rects);

/* P~ of every rectangle: out_host[j][k][d] = coefficient of w^d mod primes[k]
 * for rectangle j, d < n_terms.  Synchronises. */
int cp_sweep_read_ptilde(cp_sweep *sw, uint32_t *out_host, size_t out_len);

/* Series residues out_host[x][k][i], x = 0 bulk (square: sum alpha_i z^i of
 * Table 1; triangular: (1-x)^2 exp(f_b)/q, Baxter's product eq. (efb)),
 * x = 1 exp(f_s), x = 2 exp(f_c); modulo primes[k].  Synchronises. */
int cp_sweep_read_series(cp_sweep *sw, uint32_t *out_host, size_t out_len);

/* The three series as exact integers, CRT'd over the sweep's primes on the GPU:
 * limbs_host[(x*n_terms + i)*limbs_per_coeff + l] (limbs_len >= 3*n_terms*
 * limbs_per_coeff), series order as cp_sweep_read_series, and flags_host[x*n_terms
 * + i] (optional) as cp_crt_checked's bit 1 (the value from the first n_primes - 1
 * primes differs: not yet stable, Sec. 3.5).  Copies only the limbs (and flags)
 * to the host; synchronises.  CP_EPRIMES if any term is not stable. */
int cp_sweep_series_integers(cp_sweep *sw, uint32_t *limbs_host, size_t limbs_len, int limbs_per_coeff,
                             uint32_t *flags_host);

/* As cp_sweep_read_series into device memory, asynchronous on the sweep's stream. */
int cp_sweep_read_series_device(cp_sweep *sw, uint32_t *out_dev, size_t out_len);

/* Replace the sweep's primes (same count) for the next run: a host-to-device
 * copy of n_primes words on the sweep's stream; the tables and the graph stay. */
int cp_sweep_set_primes(cp_sweep *sw, const uint32_t *primes_host, int n_primes);

/* Run the sweep's batched gather launches once WITHOUT the graph, with a CUDA event
 * pair around each batched gather launch on the sweep's stream: *gather_ms =
 * summed gather kernel time, *n_gather = launches, *total_ms = whole pass
 * (no series kernel).  Synchronises.  For roofline measurements. */
int cp_sweep_profile(cp_sweep *sw, float *gather_ms, int *n_gather, float *total_ms);

void cp_sweep_destroy(cp_sweep *sw);

/* ---------------------------------------------------------------- serving
 * Rectangle solves of mixed lattice / L / N / primes with continuous batching.
 * Each request is solved at full degree D = L*N - 1 (Sec. 3, eq. (Z_from_T)).
 * At admission, queued requests for the same rectangle (lattice, L, N) are
 * merged into one job: one strip whose rows carry all their primes (padded to
 * a multiple of four).  The server owns one device arena of mem_budget_bytes
 * (allocated at creation) from which every admitted job takes its vectors;
 * admission is by footprint (first fit, queue order; a job that does not fit
 * yet does not block smaller ones), at most max_active jobs at once.  Each
 * step advances every active job by one per-site factor in one batched launch.
 */
typedef struct cp_server cp_server;

int cp_server_create(size_t mem_budget_bytes, int max_active, void *cuda_stream, cp_server **out);

/* Queue a solve; *req_id identifies it.  CP_ENOMEM if its footprint exceeds
 * the whole budget (it could never be admitted), CP_EINVAL on bad arguments. */
int cp_server_submit(cp_server *sv, int lattice, int L, int N, const uint32_t *primes_host, int n_primes,
                     uint64_t *req_id);

/* One step: admit queued requests that fit; one batched launch (two if some
 * rows are not 16-byte chunked) of the next per-site factor of every active
 * request (row factors, then its read-out chain); copy out and retire the
 * finished ones, returning their memory.  Synchronises the stream. */
int cp_server_step(cp_server *sv, int *n_active, int *n_queued, int *n_finished);

/* State of a request (0 queued, 1 active, 2 done, -1 failed) and, when done,
 * its residues out_host[n_primes][L*N]; times_s = {submitted, admitted,
 * finished} on the host's monotonic clock (seconds). */
int cp_server_result(cp_server *sv, uint64_t req_id, uint32_t *out_host, size_t out_len, int *state,
                     double times_s[3]);

/* Withdraw a queued (not yet admitted) request; its state becomes -1.
 * CP_EINVAL for an unknown id or a request already admitted. */
int cp_server_cancel(cp_server *sv, uint64_t req_id);

/* Ids of requests finished since the last poll (up to max_ids, oldest first). */
int cp_server_poll(cp_server *sv, uint64_t *ids_out, int max_ids, int *n_ids);

/* Forget a finished request (its result is dropped). */
int cp_server_release(cp_server *sv, uint64_t req_id);

/* Steps run, gather launches, updates (output words), free arena bytes. */
int cp_server_stats(const cp_server *sv, uint64_t *steps, uint64_t *launches, uint64_t *updates,
                    size_t *arena_free_bytes);

void cp_server_destroy(cp_server *sv);

/* Release the per-device cache of transfer-matrix tables (not in use by a
 * live strip). */
void cp_clear_table_cache(void);

const char *cp_last_error(void);

/* ---------------------------------------------------------------- diagnostics
 * Checks of the rank/unrank bijection of Sec. 3.4 on the GPU.
 * kind 0 = NCNNN partitions of m points (size M_{m-1});
 * kind 1 = square-lattice space with the pair (e, e+1) excepted (0-based e),
 *          size M_{m-1} + M_{m-2}, NCNNN ranks first (Sec. 3.4, last paragraph);
 * kind 2 = all non-crossing partitions of m <= CP_POTTS_MAX_L points (the
 *          Potts strip's space, size Catalan(m)).
 */

/* For every rank r: unrank, check canonical form and membership, rank again;
 * *n_bad = number of ranks that fail, *size = size of the space. */
int cp_debug_check_space(int kind, int m, int e, uint64_t *n_bad, uint64_t *size);

/* Launch a wait that can never complete (an mbarrier nothing arrives on),
 * bounded by `cycles` SM clock cycles, exactly like the bounded waits of the
 * TMA gather kernel; returns CP_ETIMEOUT once it has expired (the device error
 * word is read and cleared), leaving the context usable.  For testing the
 * timeout path without faulting or hanging the GPU. */
int cp_debug_wait_timeout(long long cycles);

/* The modular reduction of the gather kernels (Sec. 3.5: arithmetic modulo
 * primes below 2^31), run on the GPU on given values: out_host[k] =
 * v_host[k] mod p_host[k] in [0, p), computed exactly as the kernels reduce an
 * accumulator (integer Barrett step from the bias p 2^21, see the kernels'
 * source).  Requires 2 <= p_host[k] < 2^31 and |v_host[k]| < p_host[k] * 2^20
 * (the bound the table build enforces on every destination); CP_EINVAL
 * otherwise.  Synchronous. */
int cp_debug_reduce(const int64_t *v_host, const uint32_t *p_host, int n, uint32_t *out_host);

/* The 32-bit reduction of the bulk-copy gather (Sec. 3.5), which it uses when
 * every prime of a launch is at least 2^17: a word's sum is kept as two
 * 32-bit halves, u = hi_host[k] 2^16 + lo_host[k], and reduced from them with
 * 32-bit operations.  out_host[k] = u mod p_host[k] in [0, p) when full != 0,
 * else (u mod p) or (u mod p) - p, a signed representative in [-p, p) as the
 * kernel stores for outputs that only feed further gathers.  Requires
 * 2^17 <= p_host[k] < 2^31 and 0 < u < p_host[k] 2^16; CP_EINVAL otherwise.
 * A diagnostic (it allocates device buffers).  Synchronous. */
int cp_debug_reduce_halves(const int32_t *lo_host, const int32_t *hi_host, const uint32_t *p_host, int n, int full,
                           uint32_t *out_host);

/* One chromatic transfer-matrix table as the kernels use it (CSR by
 * destination): paired = 1 for the square lattice's two-site tables; which = 0
 * for the row factors (index 0 = T_1, or T_2 T_1 when paired), 1 for the
 * read-out chain.  info[0..3] = source states, destination states, non-zeros,
 * source bits of the packed edge (src | shift << bits | coef << (bits + 2),
 * coef in two's complement).  row_ptr_host (max_rows >= destinations + 1) and
 * edges_host (max_edges >= non-zeros) may be NULL to query info only.  Builds
 * the tables on the current device if needed. */
int cp_debug_table(int lattice, int L, int paired, int which, int index, uint32_t *row_ptr_host, uint64_t max_rows,
                   uint32_t *edges_host, uint64_t max_edges, uint64_t info[4]);

/* Partitions of the space in rank order, as canonical labels:
 * out_host[r*m + i] = block label of site i (first-occurrence order).
 * Errors: CP_EINVAL if the space has more than max_states states. */
int cp_debug_enumerate_space(int kind, int m, int e, uint8_t *out_host, uint64_t max_states, uint64_t *size);

#ifdef __cplusplus
}
#endif

#endif /* CP_TM_H */
