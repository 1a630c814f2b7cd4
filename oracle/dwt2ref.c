/*
 * dwt2ref.c -- the oracle: a plain, slow, CPU reference of the 2-D discrete
 * wavelet transform computed by separable lifting.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this code.  The GPU library shares nothing with
 * it (no headers, constants or helpers).
 *
 * What it computes (Barina et al., "Accelerating Discrete Wavelet Transforms on
 * Parallel Architectures", arXiv:1704.08657):
 *
 *   - One lifting pair is the matrix product  [1 U; 0 1] [1 0; P 1]  (Eq. 2):
 *     the predict P acts first (column vectors, rightmost matrix first), then
 *     the update U.  K pairs are applied in order.
 *   - The 2-D transform is the tensor product of 1-D transforms (Background).
 *     Separable lifting applies, for every pair, the four steps
 *     T_P^H, T_P^V, S_U^H, S_U^V in that order (the scheme
 *     "S_U^V | S_U^H | T_P^V | T_P^H", rightmost first, Background section).
 *     T_P^H adds P(c1) to c2 and P(c3) to c4 along rows, T_P^V adds P*(c1) to
 *     c3 and P*(c2) to c4 along columns, S_U^H / S_U^V likewise for U.
 *
 * Readings where the paper is silent:
 *   - CDF 9/7 lifting constants alpha..zeta (not printed in the paper): the
 *     standard values below.  Scaling: low-pass samples times zeta, high-pass
 *     samples divided by zeta, per axis.
 *   - Alignment: odd sample x[2n+1] is predicted from x[2n] and x[2n+2]; even
 *     sample x[2n] is updated from x[2n-1] and x[2n+1].
 *   - Boundary: whole-sample symmetric extension applied in every lifting step
 *     (x[-1] = x[1], x[n] = x[n-2]).
 *   - Integer CDF 5/3 (reversible): predict d = x_odd - floor((x_l + x_r)/2),
 *     update s = x_even + floor((d_l + d_r + 2)/4), same step order as above.
 *   - Layout: Mallat.  Low length ceil(n/2), high length floor(n/2).  The
 *     coefficient of sample (2i+a, 2j+b) goes to row i + a*ceil(h/2), column
 *     j + b*ceil(w/2) of the level's h x w region; the next level works on the
 *     top-left ceil(h/2) x ceil(w/2) low-low region.
 *   - Every level's input must have both sides >= 2.
 *   - DD 13/7 (Deslauriers-Dubuc interpolating wavelet, the paper's third
 *     wavelet in Table 1; its constants are not printed there): one lifting
 *     pair with the 4-tap cubic-interpolation predict
 *     d[n] = x[2n+1] - (9 (x[2n] + x[2n+2]) - (x[2n-2] + x[2n+4])) / 16 and the
 *     4-tap update s[n] = x[2n] + (9 (d[n-1] + d[n]) - (d[n-2] + d[n+1])) / 32,
 *     which multiply out to the 13-tap low-pass and 7-tap high-pass filters;
 *     no scaling step (low-pass DC gain 1).  Reflections may reach up to three
 *     samples outside a row, so these steps fold indices with the periodic
 *     whole-sample rule.
 *
 * The adjoint (not in the paper) is the product of the transposed steps in
 * reverse order; each transposed step is written as the scatter that mirrors
 * the forward step's gather, so that its correctness can be checked by eye.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define REF_OK 0
#define REF_ERR_ARG (-1)
#define REF_ERR_LEVELS (-3)
#define REF_ERR_NOMEM (-8)

/* CDF 9/7: two lifting pairs (predict, update) and the scaling constant. */
static const double k97_pred[2] = {-1.586134342, 0.882911076}; /* alpha, gamma */
static const double k97_upd[2] = {-0.052980119, 0.443506852};  /* beta, delta  */
static const double k97_zeta = 1.149604398;

/* whole-sample symmetric reflection of an index that is at most one step
 * outside [0, n): -1 -> 1 and n -> n-2 (n >= 2). */
static long ws(long k, long n) {
    if (k < 0) return -k;
    if (k >= n) return 2 * (n - 1) - k;
    return k;
}

static int64_t floordiv(int64_t a, int64_t b) {
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) q -= 1;
    return q;
}

static int check_levels(long h, long w, int levels) {
    if (h < 1 || w < 1 || levels < 0) return REF_ERR_ARG;
    for (int l = 0; l < levels; ++l) {
        if (h < 2 || w < 2) return REF_ERR_LEVELS;
        h = (h + 1) / 2;
        w = (w + 1) / 2;
    }
    return REF_OK;
}

/* ---------------------------------------------------------------- float ---- */
/* All float steps act on the h x w top-left region of an array whose rows are
 * ld elements apart.  "rows" steps run along each row (the H direction),
 * "cols" steps along each column (the V direction). */

/* predict along rows: x[r][c] += a * (x[r][c-1] + x[r][c+1]) for odd c */
static void predict_rows(double* x, long h, long w, long ld, double a) {
#pragma omp parallel for schedule(static)
    for (long r = 0; r < h; ++r) {
        double* row = x + r * ld;
        for (long c = 1; c < w; c += 2) row[c] += a * (row[c - 1] + row[ws(c + 1, w)]);
    }
}

/* update along rows: x[r][c] += b * (x[r][c-1] + x[r][c+1]) for even c */
static void update_rows(double* x, long h, long w, long ld, double b) {
#pragma omp parallel for schedule(static)
    for (long r = 0; r < h; ++r) {
        double* row = x + r * ld;
        for (long c = 0; c < w; c += 2) row[c] += b * (row[ws(c - 1, w)] + row[ws(c + 1, w)]);
    }
}

/* predict along columns: row r += a * (row r-1 + row r+1) for odd r */
static void predict_cols(double* x, long h, long w, long ld, double a) {
#pragma omp parallel for schedule(static)
    for (long r = 1; r < h; r += 2) {
        double* row = x + r * ld;
        const double* up = x + (r - 1) * ld;
        const double* dn = x + ws(r + 1, h) * ld;
        for (long c = 0; c < w; ++c) row[c] += a * (up[c] + dn[c]);
    }
}

/* update along columns: row r += b * (row r-1 + row r+1) for even r */
static void update_cols(double* x, long h, long w, long ld, double b) {
#pragma omp parallel for schedule(static)
    for (long r = 0; r < h; r += 2) {
        double* row = x + r * ld;
        const double* up = x + ws(r - 1, h) * ld;
        const double* dn = x + ws(r + 1, h) * ld;
        for (long c = 0; c < w; ++c) row[c] += b * (up[c] + dn[c]);
    }
}

/* Transposed steps (adjoint).  A forward predict along rows reads the two even
 * neighbours of every odd sample and adds to the odd sample; its transpose
 * adds a times the odd sample back to the same two (reflected) even positions.
 * Each transposed step writes only samples of the other parity than it reads,
 * so the loop order does not matter; rows (or columns) are independent. */
static void predict_rows_T(double* x, long h, long w, long ld, double a) {
#pragma omp parallel for schedule(static)
    for (long r = 0; r < h; ++r) {
        double* row = x + r * ld;
        for (long c = 1; c < w; c += 2) {
            row[c - 1] += a * row[c];
            row[ws(c + 1, w)] += a * row[c];
        }
    }
}

static void update_rows_T(double* x, long h, long w, long ld, double b) {
#pragma omp parallel for schedule(static)
    for (long r = 0; r < h; ++r) {
        double* row = x + r * ld;
        for (long c = 0; c < w; c += 2) {
            row[ws(c - 1, w)] += b * row[c];
            row[ws(c + 1, w)] += b * row[c];
        }
    }
}

/* Column transposes: serial over rows (two odd rows may scatter into the same
 * even row), vectorised along the row. */
static void predict_cols_T(double* x, long h, long w, long ld, double a) {
    for (long r = 1; r < h; r += 2) {
        const double* row = x + r * ld;
        double* up = x + (r - 1) * ld;
        double* dn = x + ws(r + 1, h) * ld;
        for (long c = 0; c < w; ++c) up[c] += a * row[c];
        for (long c = 0; c < w; ++c) dn[c] += a * row[c];
    }
}

static void update_cols_T(double* x, long h, long w, long ld, double b) {
    for (long r = 0; r < h; r += 2) {
        const double* row = x + r * ld;
        double* up = x + ws(r - 1, h) * ld;
        double* dn = x + ws(r + 1, h) * ld;
        for (long c = 0; c < w; ++c) up[c] += b * row[c];
        for (long c = 0; c < w; ++c) dn[c] += b * row[c];
    }
}

/* scale factor of sample (r, c): per axis low (even) * zeta, high (odd) / zeta */
static double scale_of(long r, long c, double z) {
    double fr = (r % 2 == 0) ? z : 1.0 / z;
    double fc = (c % 2 == 0) ? z : 1.0 / z;
    return fr * fc;
}

/* interleaved (sample order) -> Mallat (band order) within the h x w region */
static int pack_f64(double* x, long h, long w, long ld) {
    double* t = (double*)malloc(sizeof(double) * (size_t)h * (size_t)w);
    if (!t) return REF_ERR_NOMEM;
    long hl = (h + 1) / 2, wl = (w + 1) / 2;
    for (long r = 0; r < h; ++r)
        for (long c = 0; c < w; ++c)
            t[(r / 2 + (r % 2) * hl) * w + (c / 2 + (c % 2) * wl)] = x[r * ld + c];
    for (long r = 0; r < h; ++r) memcpy(x + r * ld, t + r * w, sizeof(double) * (size_t)w);
    free(t);
    return REF_OK;
}

static int unpack_f64(double* x, long h, long w, long ld) {
    double* t = (double*)malloc(sizeof(double) * (size_t)h * (size_t)w);
    if (!t) return REF_ERR_NOMEM;
    long hl = (h + 1) / 2, wl = (w + 1) / 2;
    for (long r = 0; r < h; ++r)
        for (long c = 0; c < w; ++c)
            t[r * w + c] = x[(r / 2 + (r % 2) * hl) * ld + (c / 2 + (c % 2) * wl)];
    for (long r = 0; r < h; ++r) memcpy(x + r * ld, t + r * w, sizeof(double) * (size_t)w);
    free(t);
    return REF_OK;
}

static void scale_region(double* x, long h, long w, long ld, int inverse) {
#pragma omp parallel for schedule(static)
    for (long r = 0; r < h; ++r)
        for (long c = 0; c < w; ++c) {
            double f = scale_of(r, c, k97_zeta);
            if (inverse) x[r * ld + c] /= f;
            else x[r * ld + c] *= f;
        }
}

/* One level of CDF 9/7 separable lifting on the h x w region. */
static int level97_forward(double* x, long h, long w, long ld) {
    for (int k = 0; k < 2; ++k) {
        predict_rows(x, h, w, ld, k97_pred[k]); /* T_P^H */
        predict_cols(x, h, w, ld, k97_pred[k]); /* T_P^V */
        update_rows(x, h, w, ld, k97_upd[k]);   /* S_U^H */
        update_cols(x, h, w, ld, k97_upd[k]);   /* S_U^V */
    }
    scale_region(x, h, w, ld, 0);
    return pack_f64(x, h, w, ld);
}

/* Its inverse: every step undone, in reverse order. */
static int level97_inverse(double* x, long h, long w, long ld) {
    int rc = unpack_f64(x, h, w, ld);
    if (rc) return rc;
    scale_region(x, h, w, ld, 1);
    for (int k = 1; k >= 0; --k) {
        update_cols(x, h, w, ld, -k97_upd[k]);
        update_rows(x, h, w, ld, -k97_upd[k]);
        predict_cols(x, h, w, ld, -k97_pred[k]);
        predict_rows(x, h, w, ld, -k97_pred[k]);
    }
    return REF_OK;
}

/* Its transpose: (pack * scale * prod steps)^T = prod steps^T (reversed) *
 * scale * unpack. */
static int level97_adjoint(double* x, long h, long w, long ld) {
    int rc = unpack_f64(x, h, w, ld);
    if (rc) return rc;
    scale_region(x, h, w, ld, 0);
    for (int k = 1; k >= 0; --k) {
        update_cols_T(x, h, w, ld, k97_upd[k]);
        update_rows_T(x, h, w, ld, k97_upd[k]);
        predict_cols_T(x, h, w, ld, k97_pred[k]);
        predict_rows_T(x, h, w, ld, k97_pred[k]);
    }
    return REF_OK;
}

/* ------------------------------------------------------------ DD 13/7 ---- */
/* Four-tap lifting steps: a near pair at distance 1 and a far pair at distance
 * 3 (in samples) around the updated sample, weights (near, far). */
static const double kdd_pred[2] = {-9.0 / 16.0, 1.0 / 16.0};
static const double kdd_upd[2] = {9.0 / 32.0, -1.0 / 32.0};

/* whole-sample symmetric reflection of any index into [0, n) (n >= 2) */
static long fold(long k, long n) {
    const long per = 2 * (n - 1);
    long m = k % per;
    if (m < 0) m += per;
    return m < n ? m : per - m;
}

/* x[c] += a0 (x[c-1] + x[c+1]) + a1 (x[c-3] + x[c+3]) for c = first, first+2, ...
 * along rows */
static void lift4_rows(double* x, long h, long w, long ld, long first, const double* a) {
#pragma omp parallel for schedule(static)
    for (long r = 0; r < h; ++r) {
        double* row = x + r * ld;
        for (long c = first; c < w; c += 2)
            row[c] += a[0] * (row[fold(c - 1, w)] + row[fold(c + 1, w)]) +
                      a[1] * (row[fold(c - 3, w)] + row[fold(c + 3, w)]);
    }
}

/* the same along columns, rows r = first, first+2, ... */
static void lift4_cols(double* x, long h, long w, long ld, long first, const double* a) {
#pragma omp parallel for schedule(static)
    for (long r = first; r < h; r += 2) {
        double* row = x + r * ld;
        const double* u1 = x + fold(r - 1, h) * ld;
        const double* d1 = x + fold(r + 1, h) * ld;
        const double* u3 = x + fold(r - 3, h) * ld;
        const double* d3 = x + fold(r + 3, h) * ld;
        for (long c = 0; c < w; ++c) row[c] += a[0] * (u1[c] + d1[c]) + a[1] * (u3[c] + d3[c]);
    }
}

/* One level of DD 13/7 separable lifting: T_P^H, T_P^V, S_U^H, S_U^V. */
static int level137_forward(double* x, long h, long w, long ld) {
    lift4_rows(x, h, w, ld, 1, kdd_pred);
    lift4_cols(x, h, w, ld, 1, kdd_pred);
    lift4_rows(x, h, w, ld, 0, kdd_upd);
    lift4_cols(x, h, w, ld, 0, kdd_upd);
    return pack_f64(x, h, w, ld);
}

static int level137_inverse(double* x, long h, long w, long ld) {
    int rc = unpack_f64(x, h, w, ld);
    if (rc) return rc;
    const double nu[2] = {-kdd_upd[0], -kdd_upd[1]}, np[2] = {-kdd_pred[0], -kdd_pred[1]};
    lift4_cols(x, h, w, ld, 0, nu);
    lift4_rows(x, h, w, ld, 0, nu);
    lift4_cols(x, h, w, ld, 1, np);
    lift4_rows(x, h, w, ld, 1, np);
    return REF_OK;
}

/* level sizes: sizes[l] = input side of level l (l = 0 .. levels-1) */
static void level_sides(long n, int levels, long* sides) {
    for (int l = 0; l < levels; ++l) {
        sides[l] = n;
        n = (n + 1) / 2;
    }
}

int dwt2ref_forward_f64(const double* in, double* out, long h, long w, int levels) {
    int rc = check_levels(h, w, levels);
    if (rc) return rc;
    if (!in || !out) return REF_ERR_ARG;
    if (out != in) memcpy(out, in, sizeof(double) * (size_t)h * (size_t)w);
    long hs[64], wsz[64];
    if (levels > 64) return REF_ERR_LEVELS;
    level_sides(h, levels, hs);
    level_sides(w, levels, wsz);
    for (int l = 0; l < levels; ++l) {
        rc = level97_forward(out, hs[l], wsz[l], w);
        if (rc) return rc;
    }
    return REF_OK;
}

int dwt2ref_inverse_f64(const double* coef, double* out, long h, long w, int levels) {
    int rc = check_levels(h, w, levels);
    if (rc) return rc;
    if (!coef || !out) return REF_ERR_ARG;
    if (out != coef) memcpy(out, coef, sizeof(double) * (size_t)h * (size_t)w);
    long hs[64], wsz[64];
    if (levels > 64) return REF_ERR_LEVELS;
    level_sides(h, levels, hs);
    level_sides(w, levels, wsz);
    for (int l = levels - 1; l >= 0; --l) {
        rc = level97_inverse(out, hs[l], wsz[l], w);
        if (rc) return rc;
    }
    return REF_OK;
}

int dwt2ref_adjoint_f64(const double* gcoef, double* gin, long h, long w, int levels) {
    int rc = check_levels(h, w, levels);
    if (rc) return rc;
    if (!gcoef || !gin) return REF_ERR_ARG;
    if (gin != gcoef) memcpy(gin, gcoef, sizeof(double) * (size_t)h * (size_t)w);
    long hs[64], wsz[64];
    if (levels > 64) return REF_ERR_LEVELS;
    level_sides(h, levels, hs);
    level_sides(w, levels, wsz);
    for (int l = levels - 1; l >= 0; --l) {
        rc = level97_adjoint(gin, hs[l], wsz[l], w);
        if (rc) return rc;
    }
    return REF_OK;
}

int dwt2ref_forward_dd137_f64(const double* in, double* out, long h, long w, int levels) {
    int rc = check_levels(h, w, levels);
    if (rc) return rc;
    if (!in || !out) return REF_ERR_ARG;
    if (out != in) memcpy(out, in, sizeof(double) * (size_t)h * (size_t)w);
    long hs[64], wsz[64];
    if (levels > 64) return REF_ERR_LEVELS;
    level_sides(h, levels, hs);
    level_sides(w, levels, wsz);
    for (int l = 0; l < levels; ++l) {
        rc = level137_forward(out, hs[l], wsz[l], w);
        if (rc) return rc;
    }
    return REF_OK;
}

int dwt2ref_inverse_dd137_f64(const double* coef, double* out, long h, long w, int levels) {
    int rc = check_levels(h, w, levels);
    if (rc) return rc;
    if (!coef || !out) return REF_ERR_ARG;
    if (out != coef) memcpy(out, coef, sizeof(double) * (size_t)h * (size_t)w);
    long hs[64], wsz[64];
    if (levels > 64) return REF_ERR_LEVELS;
    level_sides(h, levels, hs);
    level_sides(w, levels, wsz);
    for (int l = levels - 1; l >= 0; --l) {
        rc = level137_inverse(out, hs[l], wsz[l], w);
        if (rc) return rc;
    }
    return REF_OK;
}

/* -------------------------------------------------------------- integer ---- */
/* Reversible CDF 5/3 on int64 with floor rounding. */

static void predict_rows_i(int64_t* x, long h, long w, long ld, int sign) {
#pragma omp parallel for schedule(static)
    for (long r = 0; r < h; ++r) {
        int64_t* row = x + r * ld;
        for (long c = 1; c < w; c += 2) row[c] -= sign * floordiv(row[c - 1] + row[ws(c + 1, w)], 2);
    }
}

static void update_rows_i(int64_t* x, long h, long w, long ld, int sign) {
#pragma omp parallel for schedule(static)
    for (long r = 0; r < h; ++r) {
        int64_t* row = x + r * ld;
        for (long c = 0; c < w; c += 2) row[c] += sign * floordiv(row[ws(c - 1, w)] + row[ws(c + 1, w)] + 2, 4);
    }
}

static void predict_cols_i(int64_t* x, long h, long w, long ld, int sign) {
#pragma omp parallel for schedule(static)
    for (long r = 1; r < h; r += 2) {
        int64_t* row = x + r * ld;
        const int64_t* up = x + (r - 1) * ld;
        const int64_t* dn = x + ws(r + 1, h) * ld;
        for (long c = 0; c < w; ++c) row[c] -= sign * floordiv(up[c] + dn[c], 2);
    }
}

static void update_cols_i(int64_t* x, long h, long w, long ld, int sign) {
#pragma omp parallel for schedule(static)
    for (long r = 0; r < h; r += 2) {
        int64_t* row = x + r * ld;
        const int64_t* up = x + ws(r - 1, h) * ld;
        const int64_t* dn = x + ws(r + 1, h) * ld;
        for (long c = 0; c < w; ++c) row[c] += sign * floordiv(up[c] + dn[c] + 2, 4);
    }
}

static int pack_i64(int64_t* x, long h, long w, long ld, int unpack) {
    int64_t* t = (int64_t*)malloc(sizeof(int64_t) * (size_t)h * (size_t)w);
    if (!t) return REF_ERR_NOMEM;
    long hl = (h + 1) / 2, wl = (w + 1) / 2;
    for (long r = 0; r < h; ++r)
        for (long c = 0; c < w; ++c) {
            long pr = r / 2 + (r % 2) * hl, pc = c / 2 + (c % 2) * wl;
            if (unpack) t[r * w + c] = x[pr * ld + pc];
            else t[pr * w + pc] = x[r * ld + c];
        }
    for (long r = 0; r < h; ++r) memcpy(x + r * ld, t + r * w, sizeof(int64_t) * (size_t)w);
    free(t);
    return REF_OK;
}

int dwt2ref_forward_i64(const int64_t* in, int64_t* out, long h, long w, int levels) {
    int rc = check_levels(h, w, levels);
    if (rc) return rc;
    if (!in || !out) return REF_ERR_ARG;
    if (out != in) memcpy(out, in, sizeof(int64_t) * (size_t)h * (size_t)w);
    long hs[64], wsz[64];
    if (levels > 64) return REF_ERR_LEVELS;
    level_sides(h, levels, hs);
    level_sides(w, levels, wsz);
    for (int l = 0; l < levels; ++l) {
        long hh = hs[l], ww = wsz[l];
        predict_rows_i(out, hh, ww, w, 1); /* T_P^H */
        predict_cols_i(out, hh, ww, w, 1); /* T_P^V */
        update_rows_i(out, hh, ww, w, 1);  /* S_U^H */
        update_cols_i(out, hh, ww, w, 1);  /* S_U^V */
        rc = pack_i64(out, hh, ww, w, 0);
        if (rc) return rc;
    }
    return REF_OK;
}

int dwt2ref_inverse_i64(const int64_t* coef, int64_t* out, long h, long w, int levels) {
    int rc = check_levels(h, w, levels);
    if (rc) return rc;
    if (!coef || !out) return REF_ERR_ARG;
    if (out != coef) memcpy(out, coef, sizeof(int64_t) * (size_t)h * (size_t)w);
    long hs[64], wsz[64];
    if (levels > 64) return REF_ERR_LEVELS;
    level_sides(h, levels, hs);
    level_sides(w, levels, wsz);
    for (int l = levels - 1; l >= 0; --l) {
        long hh = hs[l], ww = wsz[l];
        rc = pack_i64(out, hh, ww, w, 1);
        if (rc) return rc;
        update_cols_i(out, hh, ww, w, -1);
        update_rows_i(out, hh, ww, w, -1);
        predict_cols_i(out, hh, ww, w, -1);
        predict_rows_i(out, hh, ww, w, -1);
    }
    return REF_OK;
}

/* number of threads the float/integer loops use */
int dwt2ref_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void dwt2ref_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
