/*
 * FP64 CPU oracle for the DPM scoring path -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the package's smoke check and the benchmark's CPU-baseline leg may load this library. It shares no
 * code with the CUDA path. Every routine is the plain definition from the paper, written as nested loops in double
 * precision over FP32 inputs; OpenMP only splits independent outputs across threads and never changes the order of a
 * sum.
 *
 *   oracle_correlate      filter response f . phi(p) at every valid placement (Sec. 2, score equation; Sec. 4, alpha)
 *   oracle_correlate_rank1 one rank-1 term ((I o c) o a) o b of the separable form (Sec. 4, the I o T identity)
 *   oracle_dt1d           1-D generalised distance transform, brute force O(n^2) (Sec. 2, argmax equation)
 *   oracle_dt2d           2-D transform as an x pass then a y pass of oracle_dt1d (Sec. 2, argmax equation)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/*
 * Valid correlation of one filter with one feature map (Sec. 2: f . phi(p); Sec. 4: alpha = N'M'NML products).
 *   feat : [H][W][L] FP32, cell (y, x) channel c at ((y*W)+x)*L+c
 *   filt : [h][w][L] FP64
 *   out  : [H-h+1][W-w+1] FP64, out[y][x] = sum_{dy<h, dx<w, c<L} filt[dy][dx][c] * feat[y+dy][x+dx][c]
 * Nothing is written when the filter does not fit.
 */
void oracle_correlate(const float *feat, int H, int W, int L, const double *filt, int h, int w, double *out)
{
    const int Ho = H - h + 1, Wo = W - w + 1;
    if (Ho <= 0 || Wo <= 0) return;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < Ho; ++y) {
        for (int x = 0; x < Wo; ++x) {
            double acc = 0.0;
            for (int dy = 0; dy < h; ++dy)
                for (int dx = 0; dx < w; ++dx)
                    for (int c = 0; c < L; ++c)
                        acc += filt[((size_t)dy * w + dx) * L + c] *
                               (double)feat[((size_t)(y + dy) * W + (x + dx)) * L + c];
            out[(size_t)y * Wo + x] = acc;
        }
    }
}

/*
 * One rank-1 term of the separable form of Sec. 4 (I o T = sum_r ((I o a_r) o b_r) o c_r), evaluated channel first:
 *   Z[y][x] = sum_c c[c] feat[y][x][c]          (correlation with the L-vector)
 *   T[y][x] = sum_dy a[dy] Z[y+dy][x]           (correlation with the h-vector along y)
 *   out[y][x] = sum_dx b[dx] T[y][x+dx]         (correlation with the w-vector along x)
 * out is [H-h+1][W-w+1]; scratch must hold H*W + (H-h+1)*W doubles.
 */
void oracle_correlate_rank1(const float *feat, int H, int W, int L, const double *a, int h, const double *b, int w,
                            const double *c, double *out, double *scratch)
{
    const int Ho = H - h + 1, Wo = W - w + 1;
    if (Ho <= 0 || Wo <= 0) return;
    double *Z = scratch, *T = scratch + (size_t)H * W;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            double acc = 0.0;
            for (int k = 0; k < L; ++k) acc += c[k] * (double)feat[((size_t)y * W + x) * L + k];
            Z[(size_t)y * W + x] = acc;
        }
    for (int y = 0; y < Ho; ++y)
        for (int x = 0; x < W; ++x) {
            double acc = 0.0;
            for (int dy = 0; dy < h; ++dy) acc += a[dy] * Z[(size_t)(y + dy) * W + x];
            T[(size_t)y * W + x] = acc;
        }
    for (int y = 0; y < Ho; ++y)
        for (int x = 0; x < Wo; ++x) {
            double acc = 0.0;
            for (int dx = 0; dx < w; ++dx) acc += b[dx] * T[(size_t)y * W + x + dx];
            out[(size_t)y * Wo + x] = acc;
        }
}

/*
 * 1-D generalised distance transform by brute force (Sec. 2, p_i = argmax_p (f_i phi(p) - d_i psi(p, p0))):
 *   D[p] = max_{0<=q<n} f[q] - (lin*(q-p) + quad*(q-p)^2),  I[p] = the smallest q attaining the maximum.
 * Every q is tried for every p (the displacement is unbounded over the map).
 */
void oracle_dt1d(const double *f, int n, double lin, double quad, double *D, int32_t *I)
{
    for (int p = 0; p < n; ++p) {
        double best = -INFINITY;
        int arg = -1;
        for (int q = 0; q < n; ++q) {
            const double dq = (double)(q - p);
            const double v = f[q] - (lin * dq + quad * dq * dq);
            if (v > best) { best = v; arg = q; }
        }
        D[p] = best;
        I[p] = arg;
    }
}

/*
 * 2-D generalised distance transform of one part score map (Sec. 2), d = coefficients of (dx, dx^2, dy, dy^2),
 * displacement = part position - anchor:
 *   D[y][x] = max_{qy,qx} S[qy][qx] - (d0*(qx-x) + d1*(qx-x)^2 + d2*(qy-y) + d3*(qy-y)^2)
 * computed as an x pass over every row then a y pass over every column (the cost is a sum of an x and a y term, so
 * the maximum splits). (Iy, Ix) is the lexicographically smallest (qy, qx) among the maximisers: the y pass keeps the
 * smallest row, and Ix is the smallest column maximising that row's x pass.
 * S, D: [H][W] FP64; Iy, Ix: [H][W] int32.
 */
void oracle_dt2d(const double *S, int H, int W, const double *d, double *D, int32_t *Iy, int32_t *Ix)
{
    double *V = (double *)malloc(sizeof(double) * (size_t)H * W);
    int32_t *IxRow = (int32_t *)malloc(sizeof(int32_t) * (size_t)H * W);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y) oracle_dt1d(S + (size_t)y * W, W, d[0], d[1], V + (size_t)y * W, IxRow + (size_t)y * W);
#pragma omp parallel for schedule(static)
    for (int x = 0; x < W; ++x) {
        double *col = (double *)malloc(sizeof(double) * (size_t)H);
        double *out = (double *)malloc(sizeof(double) * (size_t)H);
        int32_t *arg = (int32_t *)malloc(sizeof(int32_t) * (size_t)H);
        for (int y = 0; y < H; ++y) col[y] = V[(size_t)y * W + x];
        oracle_dt1d(col, H, d[2], d[3], out, arg);
        for (int y = 0; y < H; ++y) {
            D[(size_t)y * W + x] = out[y];
            Iy[(size_t)y * W + x] = arg[y];
            Ix[(size_t)y * W + x] = IxRow[(size_t)arg[y] * W + x];
        }
        free(col); free(out); free(arg);
    }
    free(V);
    free(IxRow);
}
