// Host FP64 CP-ALS (Sec. 4) used by tdpm_decompose.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

namespace tdpm {

struct CpResult {
    std::vector<double> weights;           // R
    std::vector<std::vector<double>> U;    // U[m]: dims[m] x R, row-major, unit columns
    int iters = 0;
    double rel_error = 0.0;                // ||T - CP||_F / ||T||_F after the last cycle
};

// Rank-R CP of a dense tensor T (row-major, last mode fastest) by ALS, started from the leading eigenvectors of each
// small mode unfolding (Gaussian columns beyond them, seeded).
CpResult cp_als(const double *T, const std::vector<int> &dims, int R, int max_iters, double tol, uint64_t seed);

double frob(const double *T, size_t n);

}  // namespace tdpm
