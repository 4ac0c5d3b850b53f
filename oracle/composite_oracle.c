/*
 * composite_oracle.c -- plain, slow, obviously correct CPU oracle of the
 * iterative ensemble composite (Johnson & Jankun-Kelly, "Efficacy of Images
 * Versus Data Buffers").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark call this code.  It shares no code, header or
 * table with the CUDA library and must never sit on the product path.
 *
 * What it computes, for a multiset S of flood-extent rasters, N = |S|:
 *   flood_m(p) = 1 if mask_m[p] != 0 else 0     (flood coverage images, Sec. 2, Fig. 1)
 *   count(p)   = sum over m in S of flood_m(p)  (the accumulation kernel of Fig. 2 / Fig. 3,
 *                                                step 4, applied once per member)
 *   bucket(p)  = N == 0 ? 0 : floor(255 * count(p) / N)   (overlap class, Fig. 1 caption)
 *   rgba(p)    = LUT[bucket(p)]                 (blue saturation map, Fig. 1 caption)
 *   hist[b]    = #{p : bucket(p) == b}          (frequency of overlap classes, Fig. 1 caption)
 *   mean(p)    = (1/N) sum over m in S of d_m(p), FP64, N = 0 => 0  (mean-depth composite)
 * Members may be added and removed in any order (the interactive list of
 * Fig. 1); the state after any sequence equals a recompute over the final S.
 *
 * Plain C99, no intrinsics, no threads: the loops follow the definition
 * member by member, row by row, pixel by pixel.
 */
#include <stdint.h>
#include <string.h>

/* counts[y*width + x] += sign * flood_m(x, y) for every member m of the batch.
 * members: n rasters, member m at members + m*member_stride, row y at
 * + y*row_pitch, pixel x at + x (bytes).  counts: int64[width*height].
 * sign is +1 (add) or -1 (remove).  Returns the number of pixels whose count
 * is negative afterwards (0 unless a remove took away more than was added). */
int64_t oracle_count_apply(int64_t *counts, const uint8_t *members, int64_t n,
                           int64_t width, int64_t height, int64_t row_pitch,
                           int64_t member_stride, int32_t sign)
{
    int64_t m, y, x, negative = 0;
    for (m = 0; m < n; ++m) {
        const uint8_t *member = members + m * member_stride;
        for (y = 0; y < height; ++y) {
            const uint8_t *row = member + y * row_pitch;
            for (x = 0; x < width; ++x) {
                if (row[x] != 0)
                    counts[y * width + x] += sign;
            }
        }
    }
    for (x = 0; x < width * height; ++x)
        if (counts[x] < 0)
            ++negative;
    return negative;
}

/* bucket[p] = floor(255 * count[p] / n_members), 0 when n_members == 0.
 * Exact integer arithmetic: 255 * count fits in 64 bits for any count that
 * fits in 32 bits.  Returns -1 if some count lies outside [0, n_members]. */
int32_t oracle_bucket(const int64_t *counts, int64_t n_members, int64_t npix,
                      uint8_t *bucket)
{
    int64_t p;
    for (p = 0; p < npix; ++p) {
        if (counts[p] < 0 || counts[p] > n_members)
            return -1;
        if (n_members == 0)
            bucket[p] = 0;
        else
            bucket[p] = (uint8_t)((255 * (uint64_t)counts[p]) / (uint64_t)n_members);
    }
    return 0;
}

/* rgba[4p .. 4p+3] = lut[4*bucket[p] .. 4*bucket[p]+3]. */
void oracle_rgba(const uint8_t *bucket, const uint8_t *lut, int64_t npix,
                 uint8_t *rgba)
{
    int64_t p;
    int c;
    for (p = 0; p < npix; ++p)
        for (c = 0; c < 4; ++c)
            rgba[4 * p + c] = lut[4 * (int64_t)bucket[p] + c];
}

/* hist[b] = number of pixels whose overlap class is b, b = 0..255. */
void oracle_histogram(const uint8_t *bucket, int64_t npix, uint64_t *hist)
{
    int64_t p;
    int b;
    for (b = 0; b < 256; ++b)
        hist[b] = 0;
    for (p = 0; p < npix; ++p)
        hist[bucket[p]] += 1;
}

/* The default colour table: bucket b -> (255-b, 255-b, 255, 255), white at
 * no overlap, fully saturated blue where every member floods. */
void oracle_default_lut(uint8_t *lut)
{
    int b;
    for (b = 0; b < 256; ++b) {
        lut[4 * b + 0] = (uint8_t)(255 - b);
        lut[4 * b + 1] = (uint8_t)(255 - b);
        lut[4 * b + 2] = 255;
        lut[4 * b + 3] = 255;
    }
}

/* sums[y*width + x] += sign * d_m(x, y) in FP64 for every member of the batch.
 * depths: float32 rasters, member m at depths + m*member_stride, row y at
 * + y*row_pitch (both in elements). */
void oracle_depth_apply(double *sums, const float *depths, int64_t n,
                        int64_t width, int64_t height, int64_t row_pitch,
                        int64_t member_stride, int32_t sign)
{
    int64_t m, y, x;
    for (m = 0; m < n; ++m) {
        const float *member = depths + m * member_stride;
        for (y = 0; y < height; ++y) {
            const float *row = member + y * row_pitch;
            for (x = 0; x < width; ++x)
                sums[y * width + x] += (double)sign * (double)row[x];
        }
    }
}

/* mean[p] = sums[p] / n_members, 0 when n_members == 0. */
void oracle_mean(const double *sums, int64_t n_members, int64_t npix, double *mean)
{
    int64_t p;
    for (p = 0; p < npix; ++p)
        mean[p] = n_members == 0 ? 0.0 : sums[p] / (double)n_members;
}
