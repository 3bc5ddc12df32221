// Finite-lattice series kernel (Sec. 4.1-4.3): parameters and launcher.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cp {

constexpr int kMaxSeries = 128;  // longest series (terms) handled

struct SeriesParams {
    int lattice;  // CP_SQUARE / CP_TRIANGULAR
    int k;        // finite-lattice order: rectangles with k-3 <= r+s <= k, r <= s
    int n;        // terms per series
    int D1;       // coefficients per P~ row (D+1 >= n)
    int P;        // primes
    int Pg;       // primes per group: ptilde is laid out [P/Pg][n_rects][D1][Pg]
    int n_rects;
    int mmax;     // widest strip, (k-1)/2 when the extra square-lattice term applies
    int add_mu;   // 1: add the mu_{2m} z^{4m-1} terms (square lattice, odd k)
};

// ptilde [P/Pg][n_rects][D1][Pg], rects (r, s), primes [P] -> out [3][P][n].  err |= 1 if a P~ lacks constant term 1.
int launch_flm_series(const uint32_t *ptilde, const int2 *rects, const uint32_t *primes, const SeriesParams &sp,
                      uint32_t *out, int *err, cudaStream_t st);

}  // namespace cp
