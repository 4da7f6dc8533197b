/*
 * sobel4_oracle.c — plain CPU oracle for the four-directional 5x5 Sobel operator.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA library; the product path never calls
 * it.
 *
 * What it computes (the plain definition, written out with no factoring):
 *
 *   For every pixel (y, x) and each direction k in {x, y, d, dt}
 *
 *       R_k(y, x) = sum_{i=0..4} sum_{j=0..4} K_k[i][j] * I~(y + i - 2, x + j - 2)
 *
 *   where K_k are the four integer masks of Eq. (3) (Section 3.1), applied in
 *   correlation order (mask row 0 meets input row y-2, mask column 0 meets input
 *   column x-2: the orientation of Eq. (6) and Eq. (13)), and I~ is the image
 *   under the border rule.  Then, in exact integer arithmetic,
 *
 *       S = R_x^2 + R_y^2 + R_d^2 + R_dt^2                            (Eq. 4)
 *
 *   and the gradient magnitude G = sqrt(S) of Eq. (4) is delivered as
 *     F32   : sqrtf((float)S)  (int -> fp32 round-to-nearest-even, then the
 *             IEEE-754 correctly rounded single-precision square root),
 *     U8    : min(255, round(sqrt(S))) by an exact integer rule (no float),
 *     U16   : round(sqrt(S)) by the same rule, unsaturated,
 *     EDGE8 : 255 where S >= thr (thr = ceil(T^2) for a threshold T), else 0,
 *     S16X4 : the four responses R_x, R_y, R_d, R_dt as int16 planes.
 *
 *   Border rules (Section 4.3: the kernel's output is 2r rows and columns
 *   smaller than its input; the frame is written as 0 here):
 *     0 VALID      : only 2 <= y <= H-3, 2 <= x <= W-3 are computed; every other
 *                    output pixel (all formats) is 0.
 *     1 REPLICATE  : indices clamped to the image.
 *     2 REFLECT101 : -1 -> 1, -2 -> 2, n -> n-2, n+1 -> n-3 (needs n >= 3).
 *     3 CONSTANT0  : pixels outside the image read as 0.
 *
 * Integer range: |R_k| <= 48 * 255 = 12240 and S <= 4 * 12240^2 = 599,270,400,
 * so int32 is exact everywhere.
 *
 * Build: gcc -O2 -fPIC -shared -pthread (never -ffast-math).
 */
#include <math.h>
#include <pthread.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* The four masks of Eq. (3), Section 3.1, verbatim: G_x, G_y, G_d, G_dt. */
static const int32_t ORACLE_MASKS[4][5][5] = {
    {/* G_x  (0 degrees)   */
     {-1, -2, 0, 2, 1},
     {-4, -8, 0, 8, 4},
     {-6, -12, 0, 12, 6},
     {-4, -8, 0, 8, 4},
     {-1, -2, 0, 2, 1}},
    {/* G_y  (90 degrees)  */
     {-1, -4, -6, -4, -1},
     {-2, -8, -12, -8, -2},
     {0, 0, 0, 0, 0},
     {2, 8, 12, 8, 2},
     {1, 4, 6, 4, 1}},
    {/* G_d  (45 degrees)  */
     {-6, -4, -1, -2, 0},
     {-4, -12, -8, 0, 2},
     {-1, -8, 0, 8, 1},
     {-2, 0, 8, 12, 4},
     {0, 2, 1, 4, 6}},
    {/* G_dt (135 degrees) */
     {0, -2, -1, -4, -6},
     {2, 0, -8, -12, -4},
     {1, 8, 0, -8, -1},
     {4, 12, 8, 0, -2},
     {6, 4, 1, 2, 0}},
};

enum { OR_VALID = 0, OR_REPLICATE = 1, OR_REFLECT101 = 2, OR_CONSTANT0 = 3 };
enum { OR_F32 = 0, OR_U8 = 1, OR_S16X4 = 2, OR_U16 = 3, OR_EDGE8 = 4 };
enum { OR_OK = 0, OR_ERR_INVALID = 1 };

/* Copy the Eq. (3) tables out (k, i, j order). */
int sobel4_oracle_masks(int32_t *out100) {
  if (!out100) return OR_ERR_INVALID;
  memcpy(out100, ORACLE_MASKS, sizeof(ORACLE_MASKS));
  return OR_OK;
}

/* Map a (possibly out-of-range) index into [0, n) under the border rule.
 * Returns -1 when the pixel lies outside and reads as 0 (CONSTANT0). */
static int map_index(int i, int n, int border) {
  if (i >= 0 && i < n) return i;
  switch (border) {
    case OR_REFLECT101:
      if (i < 0) return -i;
      return 2 * n - 2 - i;
    case OR_CONSTANT0:
      return -1;
    case OR_REPLICATE:
    case OR_VALID: /* VALID never reads outside for the pixels it computes */
    default:
      return i < 0 ? 0 : n - 1;
  }
}

static int32_t read_pixel(const uint8_t *src, size_t sp, int H, int W, int y, int x,
                          int border) {
  int yy = map_index(y, H, border);
  int xx = map_index(x, W, border);
  if (yy < 0 || xx < 0) return 0;
  return (int32_t)src[(size_t)yy * sp + (size_t)xx];
}

/* R_k(y, x) for the four masks (k, i, j order), straight from the definition. */
static void responses_at(const int32_t masks[4][5][5], const uint8_t *src, size_t sp, int H,
                         int W, int border, int y, int x, int32_t r[4]) {
  int k, i, j;
  for (k = 0; k < 4; ++k) r[k] = 0;
  for (i = 0; i < 5; ++i) {
    for (j = 0; j < 5; ++j) {
      int32_t v = read_pixel(src, sp, H, W, y + i - 2, x + j - 2, border);
      for (k = 0; k < 4; ++k) r[k] += masks[k][i][j] * v;
    }
  }
}

/* Under VALID only pixels at least `radius` (the masks' support radius: 2
 * for 5x5, 1 for 3x3) from every edge are computed; the frame stays 0. */
static int is_computed(int H, int W, int border, int y, int x, int radius) {
  if (border != OR_VALID) return 1;
  return y >= radius && y <= H - 1 - radius && x >= radius && x <= W - 1 - radius;
}

/* floor(sqrt(s)) for 0 <= s < 2^31 by the bit-by-bit integer method. */
static uint32_t isqrt_u32(uint32_t s) {
  uint32_t root = 0, bit = 1u << 30;
  while (bit > s) bit >>= 2;
  while (bit) {
    if (s >= root + bit) {
      s -= root + bit;
      root = (root >> 1) + bit;
    } else {
      root >>= 1;
    }
    bit >>= 2;
  }
  return root;
}

/* Nearest integer to sqrt(s); ties cannot occur for integer s. */
static uint32_t round_sqrt(int32_t s) {
  uint32_t n = isqrt_u32((uint32_t)s);
  /* sqrt(s) >= n + 1/2  <=>  s >= n^2 + n + 1/4  <=>  s > n^2 + n */
  if ((uint32_t)s > n * n + n) n += 1;
  return n;
}

/* min(255, nearest integer to sqrt(s)). */
static uint8_t magnitude_u8(int32_t s) {
  uint32_t n = round_sqrt(s);
  return (uint8_t)(n > 255u ? 255u : n);
}

typedef struct {
  const int32_t (*masks)[5][5];
  int radius;
  int64_t thr;
  const uint8_t *src;
  size_t sp;
  int H, W, border, fmt;
  void *dst;
  size_t dp;
  int y0, y1;
} band_job;

static void run_band(const band_job *jb) {
  int y, x;
  for (y = jb->y0; y < jb->y1; ++y) {
    for (x = 0; x < jb->W; ++x) {
      int32_t r[4] = {0, 0, 0, 0};
      if (is_computed(jb->H, jb->W, jb->border, y, x, jb->radius))
        responses_at(jb->masks, jb->src, jb->sp, jb->H, jb->W, jb->border, y, x, r);
      int32_t s = r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + r[3] * r[3];
      uint8_t *row = (uint8_t *)jb->dst + (size_t)y * jb->dp;
      if (jb->fmt == OR_F32) {
        ((float *)row)[x] = sqrtf((float)s);
      } else if (jb->fmt == OR_U8) {
        row[x] = magnitude_u8(s);
      } else if (jb->fmt == OR_U16) {
        ((uint16_t *)row)[x] = (uint16_t)round_sqrt(s);
      } else if (jb->fmt == OR_EDGE8) {
        /* sqrt(S) >= T  <=>  S >= T^2  <=>  S >= thr = ceil(T^2); frame 0 */
        row[x] = (is_computed(jb->H, jb->W, jb->border, y, x, jb->radius) && s >= jb->thr)
                     ? 255 : 0;
      } else {
        int k;
        for (k = 0; k < 4; ++k) {
          uint8_t *plane = (uint8_t *)jb->dst + (size_t)k * (size_t)jb->H * jb->dp;
          ((int16_t *)(plane + (size_t)y * jb->dp))[x] = (int16_t)r[k];
        }
      }
    }
  }
}

static void *band_thread(void *arg) {
  run_band((const band_job *)arg);
  return NULL;
}

static int check_args(int H, int W, int border) {
  if (H < 1 || W < 1) return OR_ERR_INVALID;
  if (border < OR_VALID || border > OR_CONSTANT0) return OR_ERR_INVALID;
  if (border == OR_REFLECT101 && (H < 3 || W < 3)) return OR_ERR_INVALID;
  return OR_OK;
}

/*
 * Gradient magnitude of an H x W u8 image (row pitch sp bytes) into dst (row
 * pitch dp bytes; S16X4 writes 4 planes at dst + k*H*dp).  Rows are split into
 * nthreads contiguous bands run on POSIX threads (nthreads <= 1: the calling
 * thread only).
 */
static int run_with(const int32_t masks[4][5][5], int radius, int64_t thr, const uint8_t *src,
                    size_t sp, int32_t H, int32_t W, int32_t border, int32_t fmt, void *dst,
                    size_t dp, int32_t nthreads);

int sobel4_oracle_run(const uint8_t *src, size_t sp, int32_t H, int32_t W, int32_t border,
                      int32_t fmt, void *dst, size_t dp, int32_t nthreads) {
  if (fmt == OR_EDGE8) return OR_ERR_INVALID; /* needs a threshold: run_masks */
  return run_with(ORACLE_MASKS, 2, 0, src, sp, H, W, border, fmt, dst, dp, nthreads);
}

/* The same with caller-supplied masks (k, i, j order, e.g. from
 * sobel4_oracle_eq5_masks) of support radius 1 or 2, and for EDGE8 the
 * threshold thr on S.  The caller keeps S = sum R_k^2 inside int32. */
int sobel4_oracle_run_masks(const int32_t *masks100, int32_t radius, int64_t thr,
                            const uint8_t *src, size_t sp, int32_t H, int32_t W, int32_t border,
                            int32_t fmt, void *dst, size_t dp, int32_t nthreads) {
  if (!masks100 || radius < 1 || radius > 2) return OR_ERR_INVALID;
  return run_with((const int32_t(*)[5][5])masks100, radius, thr, src, sp, H, W, border, fmt,
                  dst, dp, nthreads);
}

static int run_with(const int32_t masks[4][5][5], int radius, int64_t thr, const uint8_t *src,
                    size_t sp, int32_t H, int32_t W, int32_t border, int32_t fmt, void *dst,
                    size_t dp, int32_t nthreads) {
  int rc = check_args(H, W, border);
  if (rc) return rc;
  if (!src || !dst || fmt < OR_F32 || fmt > OR_EDGE8) return OR_ERR_INVALID;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > H) nthreads = H;
  band_job *jobs = (band_job *)calloc((size_t)nthreads, sizeof(band_job));
  pthread_t *tids = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
  if (!jobs || !tids) {
    free(jobs);
    free(tids);
    return OR_ERR_INVALID;
  }
  int t;
  for (t = 0; t < nthreads; ++t) {
    band_job j = {masks, radius, thr, src, sp, H, W, border, fmt, dst, dp,
                  (int)((int64_t)H * t / nthreads), (int)((int64_t)H * (t + 1) / nthreads)};
    jobs[t] = j;
  }
  for (t = 1; t < nthreads; ++t) pthread_create(&tids[t], NULL, band_thread, &jobs[t]);
  run_band(&jobs[0]);
  for (t = 1; t < nthreads; ++t) pthread_join(tids[t], NULL);
  free(jobs);
  free(tids);
  return OR_OK;
}

/*
 * The four responses as dense int32 planes out[k*H*W + y*W + x], k = x, y, d, dt.
 * Under VALID the frame is 0.
 */
int sobel4_oracle_responses(const uint8_t *src, size_t sp, int32_t H, int32_t W,
                            int32_t border, int32_t *out) {
  int rc = check_args(H, W, border);
  if (rc) return rc;
  if (!src || !out) return OR_ERR_INVALID;
  int y, x, k;
  for (y = 0; y < H; ++y) {
    for (x = 0; x < W; ++x) {
      int32_t r[4] = {0, 0, 0, 0};
      if (is_computed(H, W, border, y, x, 2))
        responses_at(ORACLE_MASKS, src, sp, H, W, border, y, x, r);
      for (k = 0; k < 4; ++k) out[(size_t)k * H * W + (size_t)y * W + x] = r[k];
    }
  }
  return OR_OK;
}

/*
 * The generalised masks of Eq. (5) (Section 3.2), written out entry by entry
 * as the four matrices are displayed there, scaled by a, each entry rounded
 * to the nearest integer.  Returns OR_ERR_INVALID when a parameter is not
 * positive, a is not an integer, or an entry is not an integer (the
 * operator requires every k_ij to be one).  (1, 2, 4, 6) gives Eq. (3).
 */
int sobel4_oracle_eq5_masks(double a, double b, double n, double m, int32_t *out100) {
  if (!out100 || !(a > 0) || !(b > 0) || !(n > 0) || !(m > 0) || a != floor(a))
    return OR_ERR_INVALID;
  const double nb = n * b, mb = m * b;
  const double K[4][5][5] = {
      {/* K_x */
       {-1, -b, 0, b, 1},
       {-n, -nb, 0, nb, n},
       {-m, -mb, 0, mb, m},
       {-n, -nb, 0, nb, n},
       {-1, -b, 0, b, 1}},
      {/* K_y */
       {-1, -n, -m, -n, -1},
       {-b, -nb, -mb, -nb, -b},
       {0, 0, 0, 0, 0},
       {b, nb, mb, nb, b},
       {1, n, m, n, 1}},
      {/* K_d */
       {-m, -n, -1, -b, 0},
       {-n, -mb, -nb, 0, b},
       {-1, -nb, 0, nb, 1},
       {-b, 0, nb, mb, n},
       {0, b, 1, n, m}},
      {/* K_dt */
       {0, -b, -1, -n, -m},
       {b, 0, -nb, -mb, -n},
       {1, nb, 0, -nb, -1},
       {n, mb, nb, 0, -b},
       {m, n, 1, b, 0}},
  };
  int k, i, j;
  for (k = 0; k < 4; ++k)
    for (i = 0; i < 5; ++i)
      for (j = 0; j < 5; ++j) {
        const double w = a * K[k][i][j];
        const double r = floor(w + 0.5);
        if (fabs(w - r) > 1e-9 * (fabs(w) > 1.0 ? fabs(w) : 1.0) || fabs(r) > 1e6)
          return OR_ERR_INVALID;
        out100[(k * 5 + i) * 5 + j] = (int32_t)r;
      }
  return OR_OK;
}

/*
 * Masks of the other operators of Section 3.1, in the 5x5 grid: op 1 = the
 * two-directional 5x5 (G_x and G_y of Eq. 3), op 2 = the two-directional
 * 3x3 of Eq. (1) as printed, centred; the diagonal masks are zero.  Returns
 * the support radius (2 or 1) through *radius.
 */
int sobel4_oracle_operator_masks(int32_t op, int32_t *out100, int32_t *radius) {
  static const int32_t G3[2][3][3] = {
      {{-1, 0, 1}, {-2, 0, 2}, {-1, 0, 1}},   /* G_x, Eq. (1) */
      {{-1, -2, -1}, {0, 0, 0}, {1, 2, 1}}};  /* G_y, Eq. (1) */
  int k, i, j;
  if (!out100 || !radius) return OR_ERR_INVALID;
  memset(out100, 0, 100 * sizeof(int32_t));
  if (op == 1) {
    memcpy(out100, ORACLE_MASKS, 2 * 25 * sizeof(int32_t));
    *radius = 2;
    return OR_OK;
  }
  if (op == 2) {
    for (k = 0; k < 2; ++k)
      for (i = 0; i < 3; ++i)
        for (j = 0; j < 3; ++j) out100[(k * 5 + 1 + i) * 5 + 1 + j] = G3[k][i][j];
    *radius = 1;
    return OR_OK;
  }
  return OR_ERR_INVALID;
}

/* sqrtf((float)s) as the oracle evaluates it, exposed for the rounding pins. */
/*
 * Grayscale from interleaved 8-bit RGB: the host-side preparation before the
 * kernel (Section 4.3), whose rule the paper leaves to another work.  The
 * reading taken here: the ITU-R BT.601 luma weights 0.299, 0.587, 0.114 in
 * 8-bit fixed point (77, 150, 29; they sum to 256), rounded half up:
 *     Y = (77 R + 150 G + 29 B + 128) >> 8.
 * Pixel x of row y is bytes 3x (R), 3x+1 (G), 3x+2 (B) of that row.
 */
int sobel4_oracle_rgb_to_gray(const uint8_t *rgb, size_t rgb_pitch, int32_t H, int32_t W,
                              uint8_t *gray, size_t gray_pitch) {
  if (!rgb || !gray || H < 1 || W < 1 || rgb_pitch < 3 * (size_t)W || gray_pitch < (size_t)W)
    return -1;
  for (int32_t y = 0; y < H; ++y) {
    const uint8_t *in = rgb + (size_t)y * rgb_pitch;
    uint8_t *out = gray + (size_t)y * gray_pitch;
    for (int32_t x = 0; x < W; ++x) {
      const uint32_t r = in[3 * x], g = in[3 * x + 1], b = in[3 * x + 2];
      out[x] = (uint8_t)((77u * r + 150u * g + 29u * b + 128u) >> 8);
    }
  }
  return 0;
}

float sobel4_oracle_magnitude_f32(int32_t s) { return sqrtf((float)s); }

/* The exact U8 rule, exposed for its pin. */
int32_t sobel4_oracle_magnitude_u8(int32_t s) { return (int32_t)magnitude_u8(s); }

/* The exact U16 rule (nearest integer to sqrt(s), unsaturated), for its pin. */
int32_t sobel4_oracle_magnitude_u16(int32_t s) { return (int32_t)round_sqrt(s); }
