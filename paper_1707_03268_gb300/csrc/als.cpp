// Host FP64 CP decomposition by alternating least squares (Sec. 4: CP form, Frobenius objective, ALS cycle).
//
// Tensors are dense, row-major with the last mode fastest. One ALS cycle replaces factor n = 0, 1, ..., N-1 in turn
// by the exact least-squares minimiser with the other factors fixed: U_n G = M with
// G = Hadamard_{m != n} (U_m^T U_m) and M = T_(n) (Khatri-Rao_{m != n} U_m) (the MTTKRP), solved by Cholesky
// (a relative ridge of 1e-12 trace(G), grown on failure, when G is singular). Scale is moved into factor 0 after
// every cycle, which leaves the model unchanged. The cycle stops after max_iters or when the residual
// ||T - CP||_F changed by at most tol * ||T||_F.
#include "als.h"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace tdpm {
namespace {

uint64_t splitmix64(uint64_t &s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double uniform01(uint64_t &s) { return ((double)(splitmix64(s) >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

double normal01(uint64_t &s)
{
    const double u1 = uniform01(s), u2 = uniform01(s);
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

// In-place lower Cholesky of an R x R SPD matrix; false if not positive definite.
bool cholesky(std::vector<double> &G, int R)
{
    for (int j = 0; j < R; ++j) {
        double d = G[j * R + j];
        for (int k = 0; k < j; ++k) d -= G[j * R + k] * G[j * R + k];
        if (!(d > 0.0)) return false;
        d = std::sqrt(d);
        G[j * R + j] = d;
        for (int i = j + 1; i < R; ++i) {
            double v = G[i * R + j];
            for (int k = 0; k < j; ++k) v -= G[i * R + k] * G[j * R + k];
            G[i * R + j] = v / d;
        }
    }
    return true;
}

// Solve (L L^T) x = b in place.
void chol_solve(const std::vector<double> &L, int R, double *b)
{
    for (int i = 0; i < R; ++i) {
        double v = b[i];
        for (int k = 0; k < i; ++k) v -= L[i * R + k] * b[k];
        b[i] = v / L[i * R + i];
    }
    for (int i = R - 1; i >= 0; --i) {
        double v = b[i];
        for (int k = i + 1; k < R; ++k) v -= L[k * R + i] * b[k];
        b[i] = v / L[i * R + i];
    }
}

struct Shape {
    std::vector<int> dims;
    size_t size = 1, outer = 1;
    int last = 0;
    explicit Shape(const std::vector<int> &d) : dims(d)
    {
        for (int v : d) size *= (size_t)v;
        last = d.back();
        outer = size / (size_t)last;
    }
};

// Decode the outer (all but last mode) linear index into a multi-index.
void decode_outer(const Shape &S, size_t o, int *idx)
{
    const int N = (int)S.dims.size();
    for (int m = N - 2; m >= 0; --m) {
        idx[m] = (int)(o % (size_t)S.dims[m]);
        o /= (size_t)S.dims[m];
    }
}

void mttkrp(const double *T, const Shape &S, const std::vector<std::vector<double>> &U, int R, int n,
            std::vector<double> &M)
{
    const int N = (int)S.dims.size();
    M.assign((size_t)S.dims[n] * R, 0.0);
    std::vector<double> P(R), Wv(R);
    int idx[8];
    const std::vector<double> &UL = U[N - 1];
    for (size_t o = 0; o < S.outer; ++o) {
        decode_outer(S, o, idx);
        std::fill(P.begin(), P.end(), 1.0);
        for (int m = 0; m < N - 1; ++m) {
            if (m == n) continue;
            const double *u = &U[m][(size_t)idx[m] * R];
            for (int r = 0; r < R; ++r) P[r] *= u[r];
        }
        const double *t = T + o * (size_t)S.last;
        if (n == N - 1) {
            for (int l = 0; l < S.last; ++l) {
                const double tv = t[l];
                double *mrow = &M[(size_t)l * R];
                for (int r = 0; r < R; ++r) mrow[r] += tv * P[r];
            }
        } else {
            std::fill(Wv.begin(), Wv.end(), 0.0);
            for (int l = 0; l < S.last; ++l) {
                const double tv = t[l];
                const double *u = &UL[(size_t)l * R];
                for (int r = 0; r < R; ++r) Wv[r] += tv * u[r];
            }
            double *mrow = &M[(size_t)idx[n] * R];
            for (int r = 0; r < R; ++r) mrow[r] += P[r] * Wv[r];
        }
    }
}

double residual(const double *T, const Shape &S, const std::vector<std::vector<double>> &U, int R)
{
    const int N = (int)S.dims.size();
    std::vector<double> P(R);
    int idx[8];
    double e2 = 0.0;
    for (size_t o = 0; o < S.outer; ++o) {
        decode_outer(S, o, idx);
        std::fill(P.begin(), P.end(), 1.0);
        for (int m = 0; m < N - 1; ++m) {
            const double *u = &U[m][(size_t)idx[m] * R];
            for (int r = 0; r < R; ++r) P[r] *= u[r];
        }
        const double *t = T + o * (size_t)S.last;
        for (int l = 0; l < S.last; ++l) {
            const double *u = &U[N - 1][(size_t)l * R];
            double x = 0.0;
            for (int r = 0; r < R; ++r) x += P[r] * u[r];
            const double d = t[l] - x;
            e2 += d * d;
        }
    }
    return std::sqrt(e2);
}

// Eigenvectors of a small symmetric matrix (cyclic Jacobi rotations), columns sorted by decreasing eigenvalue.
void sym_eig(std::vector<double> A, int n, std::vector<double> &vecs)
{
    vecs.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) vecs[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += A[(size_t)p * n + q] * A[(size_t)p * n + q];
        if (off < 1e-30) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[(size_t)p * n + q];
                if (std::fabs(apq) < 1e-300) continue;
                const double theta = (A[(size_t)q * n + q] - A[(size_t)p * n + p]) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {
                    const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = vecs[(size_t)k * n + p], vkq = vecs[(size_t)k * n + q];
                    vecs[(size_t)k * n + p] = c * vkp - s * vkq;
                    vecs[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return A[(size_t)a * n + a] > A[(size_t)b * n + b]; });
    std::vector<double> sorted((size_t)n * n);
    for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j) sorted[(size_t)k * n + j] = vecs[(size_t)k * n + order[j]];
    vecs.swap(sorted);
}

// Starting factors: for modes of at most 64 rows the leading eigenvectors of T_(m) T_(m)^T (the higher-order SVD
// subspace), Gaussian columns beyond the mode's size and for larger modes.
void init_factors(const double *T, const Shape &S, int R, uint64_t &st, std::vector<std::vector<double>> &U)
{
    const int N = (int)S.dims.size();
    for (int m = 0; m < N; ++m) {
        const int n = S.dims[m];
        U[m].resize((size_t)n * R);
        for (double &v : U[m]) v = normal01(st);
        if (n > 64) continue;
        // Gram matrix of the mode-m unfolding
        std::vector<double> G((size_t)n * n, 0.0);
        size_t inner = 1;
        for (int k = m + 1; k < N; ++k) inner *= (size_t)S.dims[k];
        const size_t outer = S.size / (inner * n);
        for (size_t o = 0; o < outer; ++o)
            for (int a = 0; a < n; ++a) {
                const double *ra = T + (o * n + a) * inner;
                for (int b = a; b < n; ++b) {
                    const double *rb = T + (o * n + b) * inner;
                    double v = 0.0;
                    for (size_t i = 0; i < inner; ++i) v += ra[i] * rb[i];
                    G[(size_t)a * n + b] += v;
                }
            }
        for (int a = 0; a < n; ++a)
            for (int b = 0; b < a; ++b) G[(size_t)a * n + b] = G[(size_t)b * n + a];
        std::vector<double> V;
        sym_eig(G, n, V);
        for (int r = 0; r < std::min(R, n); ++r)
            for (int i = 0; i < n; ++i) U[m][(size_t)i * R + r] = V[(size_t)i * n + r];
    }
}

}  // namespace

CpResult cp_als(const double *T, const std::vector<int> &dims, int R, int max_iters, double tol, uint64_t seed)
{
    const Shape S(dims);
    const int N = (int)dims.size();
    CpResult res;
    res.U.resize(N);
    uint64_t st = seed * 0x2545F4914F6CDD1Dull + 0x1234567ull;
    init_factors(T, S, R, st, res.U);
    double normT = 0.0;
    for (size_t i = 0; i < S.size; ++i) normT += T[i] * T[i];
    normT = std::sqrt(normT);

    std::vector<double> G((size_t)R * R), Gm((size_t)R * R), M, Lc;
    double f_prev = -1.0, f = normT;
    int it = 0;
    for (; it < max_iters; ++it) {
        for (int n = 0; n < N; ++n) {
            std::fill(G.begin(), G.end(), 1.0);
            for (int m = 0; m < N; ++m) {
                if (m == n) continue;
                const std::vector<double> &Um = res.U[m];
                for (int r = 0; r < R; ++r)
                    for (int s = 0; s < R; ++s) {
                        double v = 0.0;
                        for (int i = 0; i < dims[m]; ++i) v += Um[(size_t)i * R + r] * Um[(size_t)i * R + s];
                        Gm[r * R + s] = v;
                    }
                for (size_t k = 0; k < G.size(); ++k) G[k] *= Gm[k];
            }
            mttkrp(T, S, res.U, R, n, M);
            double tr = 0.0;
            for (int r = 0; r < R; ++r) tr += G[r * R + r];
            double ridge = 0.0;
            for (int attempt = 0; attempt < 40; ++attempt) {
                Lc = G;
                for (int r = 0; r < R; ++r) Lc[r * R + r] += ridge;
                if (cholesky(Lc, R)) break;
                ridge = (ridge == 0.0) ? 1e-12 * (tr > 0 ? tr : 1.0) : ridge * 10.0;
            }
            std::vector<double> &Un = res.U[n];
            for (int i = 0; i < dims[n]; ++i) {
                double *row = &M[(size_t)i * R];
                chol_solve(Lc, R, row);
                std::memcpy(&Un[(size_t)i * R], row, sizeof(double) * R);
            }
        }
        for (int m = 1; m < N; ++m) {
            for (int r = 0; r < R; ++r) {
                double nr = 0.0;
                for (int i = 0; i < dims[m]; ++i) nr += res.U[m][(size_t)i * R + r] * res.U[m][(size_t)i * R + r];
                nr = std::sqrt(nr);
                if (nr == 0.0) continue;
                for (int i = 0; i < dims[m]; ++i) res.U[m][(size_t)i * R + r] /= nr;
                for (int i = 0; i < dims[0]; ++i) res.U[0][(size_t)i * R + r] *= nr;
            }
        }
        f = residual(T, S, res.U, R);
        if (f_prev >= 0.0 && std::fabs(f_prev - f) <= tol * normT) { ++it; break; }
        if (f <= 1e-15 * normT) { ++it; break; }
        f_prev = f;
    }
    res.weights.assign(R, 1.0);
    for (int r = 0; r < R; ++r) {
        double nr = 0.0;
        for (int i = 0; i < dims[0]; ++i) nr += res.U[0][(size_t)i * R + r] * res.U[0][(size_t)i * R + r];
        nr = std::sqrt(nr);
        res.weights[r] = nr;
        if (nr > 0.0)
            for (int i = 0; i < dims[0]; ++i) res.U[0][(size_t)i * R + r] /= nr;
    }
    res.iters = it;
    res.rel_error = normT > 0 ? f / normT : 0.0;
    return res;
}

double frob(const double *T, size_t n)
{
    double s = 0.0;
    for (size_t i = 0; i < n; ++i) s += T[i] * T[i];
    return std::sqrt(s);
}

}  // namespace tdpm
