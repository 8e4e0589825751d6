/*
 * iqa_oracle.c -- plain FP64 CPU oracle for the tile-wise LISI / augLISI maps.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may load, link or call
 * this file: only the tests, the smoke check and the benchmark's CPU-baseline leg
 * use it.  It shares no code, header or constant with the CUDA library.
 *
 * What it computes (arxiv 2501.10653, "GPU Accelerated Image Quality
 * Assessment-Based Software for Transient Detection"):
 *
 *   Section 2: negative pixels of both images are set to zero, then each N x N
 *   image is cut into N_T x N_T tiles; every tile gets one LISI (Eq. 1) and one
 *   augLISI (Eq. 2) value, computed over the pixels of that tile only.
 *
 *   Eq. 1   LISI    = D * sum_i |x_i + y_i| / (|x_i - y_i| + C1)
 *                       / ( max(sum_i x_i, sum_i y_i) + C2 )
 *   Eq. 2   augLISI = 1 - sum_i |x_i + y_i| |x_i - y_i|
 *                       / ( sum_i x_i + sum_i y_i + C )
 *
 * Readings of the paper taken here (the paper does not fix them):
 *   - the clamp is "v > 0 ? v : 0", so NaN and -0 become +0;
 *   - tile t sits at tile-row r = t / (N/N_T), tile-column c = t % (N/N_T),
 *     rows counted in memory order (row-major arrays);
 *   - N_T must divide N;
 *   - D is a free constant supplied by the caller.
 *
 * Every sum is a plain sequential FP64 loop over the tile's pixels in row-major
 * order.  Build with -O2 -ffp-contract=off (no fast-math) so the arithmetic is
 * exactly what is written.  The optional OpenMP pragma only spreads whole tiles
 * over threads; it does not change any tile's arithmetic.
 */
#include <math.h>
#include <stddef.h>

/* Section 2 pre-processing: negative pixel values become zero. */
static double clamp_negative(float v)
{
    return v > 0.0f ? (double)v : 0.0;
}

/*
 * The four per-tile sums that Eq. 1 and Eq. 2 are built from, for the tile at
 * tile-row r and tile-column c:
 *   out[0] = A  = sum |x+y| / (|x-y| + C1)     (Eq. 1 numerator sum)
 *   out[1] = B  = sum |x+y| * |x-y|            (Eq. 2 numerator sum)
 *   out[2] = Sx = sum x
 *   out[3] = Sy = sum y
 * x and y are clamped before any term is formed.
 */
static void tile_sums(const float *x, const float *y, long N, long NT,
                      long r, long c, double C1, double out[4])
{
    double A = 0.0, B = 0.0, Sx = 0.0, Sy = 0.0;
    for (long i = 0; i < NT; ++i) {
        for (long j = 0; j < NT; ++j) {
            long idx = (r * NT + i) * N + (c * NT + j);
            double xi = clamp_negative(x[idx]);
            double yi = clamp_negative(y[idx]);
            double s = fabs(xi + yi);
            double d = fabs(xi - yi);
            A += s / (d + C1);
            B += s * d;
            Sx += xi;
            Sy += yi;
        }
    }
    out[0] = A;
    out[1] = B;
    out[2] = Sx;
    out[3] = Sy;
}

static int bad_shape(long N, long NT)
{
    return N < 1 || NT < 1 || NT > N || (N % NT) != 0;
}

/*
 * Per-tile sums for a list of tiles (tiles == NULL means every tile, in order
 * t = 0 .. n-1).  sums receives 4 doubles per listed tile.  threads > 1 spreads
 * tiles over OpenMP threads when the build has OpenMP.
 * Returns 0, or -1 on a bad shape or a tile index out of range.
 */
int iqa_oracle_tile_sums(const float *x, const float *y, long N, long NT,
                         double C1, const long *tiles, long ntiles,
                         double *sums, int threads)
{
    if (bad_shape(N, NT))
        return -1;
    long tiles_per_row = N / NT;
    long n = tiles_per_row * tiles_per_row;
    long count = tiles ? ntiles : n;
    for (long k = 0; k < count; ++k)
        if (tiles && (tiles[k] < 0 || tiles[k] >= n))
            return -1;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads > 0 ? threads : 1) if (threads > 1)
#endif
    for (long k = 0; k < count; ++k) {
        long t = tiles ? tiles[k] : k;
        tile_sums(x, y, N, NT, t / tiles_per_row, t % tiles_per_row, C1,
                  sums + 4 * k);
    }
    (void)threads;
    return 0;
}

/*
 * Eq. 1 and Eq. 2 for every tile.  lisi, aug: n doubles each (either may be
 * NULL); sums: n*4 doubles (may be NULL).  Returns 0, or -1 on a bad shape.
 */
int iqa_oracle_maps(const float *x, const float *y, long N, long NT,
                    double C1, double C2, double C, double D,
                    double *lisi, double *aug, double *sums, int threads)
{
    if (bad_shape(N, NT))
        return -1;
    long tiles_per_row = N / NT;
    long n = tiles_per_row * tiles_per_row;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads > 0 ? threads : 1) if (threads > 1)
#endif
    for (long t = 0; t < n; ++t) {
        double s[4];
        tile_sums(x, y, N, NT, t / tiles_per_row, t % tiles_per_row, C1, s);
        double A = s[0], B = s[1], Sx = s[2], Sy = s[3];
        if (lisi)
            lisi[t] = D * A / (fmax(Sx, Sy) + C2);          /* Eq. 1 */
        if (aug)
            aug[t] = 1.0 - B / (Sx + Sy + C);                /* Eq. 2 */
        if (sums) {
            sums[4 * t + 0] = A;
            sums[4 * t + 1] = B;
            sums[4 * t + 2] = Sx;
            sums[4 * t + 3] = Sy;
        }
    }
    (void)threads;
    return 0;
}

/* 1 when compiled with OpenMP (tiles spread over threads), else 0. */
int iqa_oracle_has_openmp(void)
{
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}
