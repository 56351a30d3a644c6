/*
 * flic_oracle.c — plain, slow, sequential CPU oracle of the FLIC hot path
 * (Hasecke, Hahn & Kummert, "FLIC: Fast Lidar Image Clustering", arXiv 2003.00575).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg may load or call this code.  It shares no code, header, table generator
 * or constant with the CUDA path; it is compiled separately with plain gcc
 * (-O2 -ffp-contract=off -fno-fast-math) so that every fp32 operation is one IEEE
 * round-to-nearest operation, never fused.
 *
 * What it computes (each function cites the passage it follows):
 *   oracle_tables     the pre-computed cosine constants of Eq. 3 (§III-B), one per row
 *                     and offset, in the form K = 2 - 2 cos(alpha) = 4 sin^2(alpha/2)
 *   oracle_pred       the thresholded squared law-of-cosines distance (Eq. 2, Eq. 3)
 *   oracle_edges      the edge bits of every pixel for offsets 1..S (§III-B-1 binary
 *                     images; §III-B-2 Map Connections with the angle scaled by offset)
 *   oracle_label      connected-component labelling by breadth-first search, one
 *                     component at a time in raster order (§III-B-1), label = min index
 *   oracle_flips      FP64 decision of every candidate pair against the fp32 one
 *   oracle_flips_paper_form
 *                     the same for the literal form of Eq. 3 (a diagnostic)
 *   oracle_project    spherical projection of xyz points into the range image (§I)
 *   oracle_scatter    labels back onto the points (§I, Fig. 1)
 *   oracle_ground     ground extraction by the angle to the reading above (§III-A, Eq. 1
 *                     in its tangent form), with the optional height-line exception
 *   oracle_edges_ex,  the same with the paper's sparse Map Connection (§III-B-2): besides
 *   oracle_label_ex   the direct neighbours, only every S-th point in each direction is
 *                     joined, to the S-th point further on (a sub-lattice map)
 *   oracle_tables_diag, oracle_label_diag
 *                     Map Connections along the diagonals of the range image (§III-B-2,
 *                     "MCs along the main diagonal"): besides the row and column offsets
 *                     1..S, pixel (r, c) is joined to (r+k, c+k) and (r+k, c-k), k = 1..S,
 *                     with the constant of the true angle between the two beams
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* A range reading is a measurement iff it is positive and finite; zero is "no return"
 * (§III-A: zero values are removed as invalid). */
static int oracle_valid(float x) { return x > 0.0f && x <= FLT_MAX; }

/*
 * Eq. 3 constant.  alpha is the angle between the two beams: for rows r and r+k at the
 * same azimuth it is the difference of their channel elevations (§III-A lookup table of
 * channel angles); for columns k apart it is k times the horizontal step supplied by the
 * manufacturer (§III-B), the angle "adjusted to the given offset" (§III-B-2).
 * Kv[r*S + k-1] (0 when r+k >= R) and Kh[r*S + k-1], k = 1..S.
 */
void oracle_tables_ex(int32_t R, const double* elev, double az_step, int32_t S, int32_t exact_ray,
                      float* Kv, float* Kh);

void oracle_tables(int32_t R, const double* elev, double az_step, int32_t S, float* Kv,
                   float* Kh) {
    oracle_tables_ex(R, elev, az_step, S, 0, Kv, Kh);
}

/*
 * exact_ray != 0: the horizontal angle is the true angle between the two rays of row r,
 * k columns apart, instead of k times the azimuth step: cos(alpha) = cos^2(e) cos(k step)
 * + sin^2(e), so K = 2 - 2 cos(alpha) = 4 cos^2(e) sin^2(k step / 2) (the paper takes the
 * manufacturer's step as the angle, §III-B; this is the variant §III-B-2's "adjusting the
 * angle to the given offset" allows for rays off the horizon).
 */
void oracle_tables_ex(int32_t R, const double* elev, double az_step, int32_t S, int32_t exact_ray,
                      float* Kv, float* Kh) {
    for (int32_t r = 0; r < R; ++r) {
        for (int32_t k = 1; k <= S; ++k) {
            float kv = 0.0f;
            if (r + k < R) {
                double alpha = fabs(elev[r + k] - elev[r]);
                double s = sin(alpha / 2.0);
                kv = (float)(4.0 * s * s);
            }
            double alpha_h = (double)k * az_step;
            double sh = sin(alpha_h / 2.0);
            double ce = exact_ray ? cos(elev[r]) : 1.0;
            Kv[r * S + (k - 1)] = kv;
            Kh[r * S + (k - 1)] = (float)(4.0 * ce * ce * sh * sh);
        }
    }
}

/*
 * Eq. 2 squared, written as D^2 = (d1 - d2)^2 + K * (d1 * d2) with K = 2 - 2 cos(alpha):
 * algebraically the expression of Eq. 3, without its cancellation of two ~d^2 terms.
 * The pair is close enough iff D^2 <= delta^2 (§III-B: one distance threshold).
 */
int32_t oracle_pred(float a, float b, float K, float delta2) {
    float t = a - b;
    float tt = t * t;
    float ab = a * b;
    float kab = K * ab;
    float d2 = tt + kab;
    return d2 <= delta2 ? 1 : 0;
}

/* The same test in the literal form of Eq. 3, d1*d1 + d2*d2 - (2 cos alpha)*d1*d2,
 * with C2 = (float)(2 cos alpha).  Diagnostic only (its cancellation is what the form
 * above removes). */
int32_t oracle_pred_paper_form(float a, float b, float C2, float delta2) {
    float aa = a * a;
    float bb = b * b;
    float ab = a * b;
    float c = C2 * ab;
    float d2 = (aa + bb) - c;
    return d2 <= delta2 ? 1 : 0;
}

static float oracle_delta2(float delta) { return delta * delta; }

/*
 * Edge bits of every pixel (§III-B-1: the binary images of horizontal and vertical
 * connections; §III-B-2: the same test repeated at offsets 1..S).  Pixel p = r*C + c:
 * bit k-1 = edge to (r, (c+k) mod C) (no wrap: only when c+k < C),
 * bit 8+k-1 = edge to (r+k, c) when r+k < R.
 */
/*
 * Which offsets a pixel's pairs may use.  Offsets 1..S from every pixel is the general
 * reading of §III-B-2.  With lattice != 0 it is the paper's sparse map instead: the
 * direct neighbours (offset 1) of every pixel, and offset S only from the points of the
 * sub-lattice of every S-th row and every S-th column ("connecting only every n-th
 * point", with n = S); (r, c) is the pair's left or upper end, c its column before any
 * wrap.
 */
static int oracle_offset_used(int32_t lattice, int32_t S, int32_t k, int32_t r, int32_t c) {
    if (!lattice || k == 1) return 1;
    return k == S && r % S == 0 && c % S == 0;
}

void oracle_edges_ex(int32_t R, int32_t C, const float* range, const float* Kv, const float* Kh,
                     int32_t S, float delta, int32_t wrap, int32_t lattice, uint16_t* mask);

void oracle_edges(int32_t R, int32_t C, const float* range, const float* Kv, const float* Kh,
                  int32_t S, float delta, int32_t wrap, uint16_t* mask) {
    oracle_edges_ex(R, C, range, Kv, Kh, S, delta, wrap, 0, mask);
}

void oracle_edges_ex(int32_t R, int32_t C, const float* range, const float* Kv, const float* Kh,
                     int32_t S, float delta, int32_t wrap, int32_t lattice, uint16_t* mask) {
    float delta2 = oracle_delta2(delta);
    for (int32_t r = 0; r < R; ++r) {
        for (int32_t c = 0; c < C; ++c) {
            uint16_t m = 0;
            float a = range[(int64_t)r * C + c];
            if (oracle_valid(a)) {
                for (int32_t k = 1; k <= S; ++k) {
                    if (!oracle_offset_used(lattice, S, k, r, c)) continue;
                    int32_t cc = c + k;
                    int has = 1;
                    if (cc >= C) {
                        if (wrap) cc = cc % C; else has = 0;
                    }
                    if (has) {
                        float b = range[(int64_t)r * C + cc];
                        if (oracle_valid(b) && oracle_pred(a, b, Kh[r * S + k - 1], delta2))
                            m |= (uint16_t)(1u << (k - 1));
                    }
                    if (r + k < R) {
                        float b = range[(int64_t)(r + k) * C + c];
                        if (oracle_valid(b) && oracle_pred(a, b, Kv[r * S + k - 1], delta2))
                            m |= (uint16_t)(1u << (8 + k - 1));
                    }
                }
            }
            mask[(int64_t)r * C + c] = m;
        }
    }
}

/*
 * Connected-component labelling of the pixel graph (§III-B-1), "one component at a
 * time": scan pixels in raster order; an unlabelled valid pixel starts a new component
 * whose label is its own index (so each label is the minimum index of its component);
 * a breadth-first search then labels every pixel joined to it by an edge.  From pixel
 * (r,c) the candidate neighbours are (r, c+-k) (mod C with wrap) and (r+-k, c) for
 * k = 1..S; a horizontal pair uses Kh of the shared row, a vertical pair Kv of the upper
 * (smaller) row, each with the offset k that reaches it.
 * Returns the number of components, or -1 if memory for the queue is unavailable.
 */
int64_t oracle_label_ex(int32_t R, int32_t C, const float* range, const float* Kv,
                        const float* Kh, int32_t S, float delta, int32_t wrap, int32_t lattice,
                        int32_t* labels);

int64_t oracle_label(int32_t R, int32_t C, const float* range, const float* Kv, const float* Kh,
                     int32_t S, float delta, int32_t wrap, int32_t* labels) {
    return oracle_label_ex(R, C, range, Kv, Kh, S, delta, wrap, 0, labels);
}

/* oracle_label with the pairs restricted by oracle_offset_used (lattice != 0: the sparse
 * Map Connection of §III-B-2). */
int64_t oracle_label_ex(int32_t R, int32_t C, const float* range, const float* Kv,
                        const float* Kh, int32_t S, float delta, int32_t wrap, int32_t lattice,
                        int32_t* labels) {
    int64_t N = (int64_t)R * C;
    float delta2 = oracle_delta2(delta);
    int32_t* queue = (int32_t*)malloc((size_t)(N > 0 ? N : 1) * sizeof(int32_t));
    if (!queue) return -1;
    for (int64_t p = 0; p < N; ++p) labels[p] = -1;
    int64_t ncomp = 0;
    for (int64_t p0 = 0; p0 < N; ++p0) {
        if (labels[p0] != -1 || !oracle_valid(range[p0])) continue;
        ++ncomp;
        int64_t head = 0, tail = 0;
        labels[p0] = (int32_t)p0;
        queue[tail++] = (int32_t)p0;
        while (head < tail) {
            int32_t u = queue[head++];
            int32_t ur = u / C, uc = u % C;
            float a = range[u];
            for (int32_t k = 1; k <= S; ++k) {
                /* horizontal, both directions */
                for (int dir = -1; dir <= 1; dir += 2) {
                    int32_t vc = uc + dir * k;
                    if (vc < 0 || vc >= C) {
                        if (!wrap) continue;
                        vc = ((vc % C) + C) % C;
                    }
                    /* the left end: u itself, or v when v lies k columns to the left */
                    if (!oracle_offset_used(lattice, S, k, ur, dir > 0 ? uc : vc)) continue;
                    int32_t v = ur * C + vc;
                    if (labels[v] != -1) continue;
                    float b = range[v];
                    if (oracle_valid(b) && oracle_pred(a, b, Kh[ur * S + k - 1], delta2)) {
                        labels[v] = (int32_t)p0;
                        queue[tail++] = v;
                    }
                }
                /* vertical, both directions; K indexed by the upper row */
                for (int dir = -1; dir <= 1; dir += 2) {
                    int32_t vr = ur + dir * k;
                    if (vr < 0 || vr >= R) continue;
                    int32_t v = vr * C + uc;
                    if (labels[v] != -1) continue;
                    int32_t top = dir > 0 ? ur : vr;
                    if (!oracle_offset_used(lattice, S, k, top, uc)) continue;
                    float b = range[v];
                    if (oracle_valid(b) && oracle_pred(a, b, Kv[top * S + k - 1], delta2)) {
                        labels[v] = (int32_t)p0;
                        queue[tail++] = v;
                    }
                }
            }
        }
    }
    free(queue);
    return ncomp;
}

/*
 * FP64 cross-check of the fp32 decision.  For every candidate pair (both readings valid)
 * D is evaluated by Eq. 2 in double with the exact angle, as
 * D = sqrt((a-b)^2 + 4ab sin^2(alpha/2)), and compared with delta (the fp32 value,
 * widened).  Counts pairs whose decision differs from the fp32 predicate and reports the
 * largest |D - delta| among them.  out[0] = candidate pairs, out[1] = flips;
 * max_dev[0] = largest |D - delta| over flips (0 if none).
 */
void oracle_flips(int32_t R, int32_t C, const float* range, const double* elev, double az_step,
                  const float* Kv, const float* Kh, int32_t S, float delta, int32_t wrap,
                  int64_t* out, double* max_dev) {
    float delta2 = oracle_delta2(delta);
    double d64 = (double)delta;
    int64_t pairs = 0, flips = 0;
    double worst = 0.0;
    for (int32_t r = 0; r < R; ++r) {
        for (int32_t c = 0; c < C; ++c) {
            float a = range[(int64_t)r * C + c];
            if (!oracle_valid(a)) continue;
            for (int32_t k = 1; k <= S; ++k) {
                for (int vert = 0; vert <= 1; ++vert) {
                    int32_t rr = r, cc = c;
                    double alpha;
                    float K;
                    if (vert) {
                        rr = r + k;
                        if (rr >= R) continue;
                        alpha = fabs(elev[rr] - elev[r]);
                        K = Kv[r * S + k - 1];
                    } else {
                        cc = c + k;
                        if (cc >= C) {
                            if (!wrap) continue;
                            cc = cc % C;
                        }
                        alpha = (double)k * az_step;
                        K = Kh[r * S + k - 1];
                    }
                    float b = range[(int64_t)rr * C + cc];
                    if (!oracle_valid(b)) continue;
                    ++pairs;
                    int f32 = oracle_pred(a, b, K, delta2);
                    double da = (double)a, db = (double)b;
                    double sa = sin(alpha / 2.0);
                    double D = sqrt((da - db) * (da - db) + 4.0 * da * db * sa * sa);
                    int f64 = D <= d64 ? 1 : 0;
                    if (f32 != f64) {
                        ++flips;
                        double dev = fabs(D - d64);
                        if (dev > worst) worst = dev;
                    }
                }
            }
        }
    }
    out[0] = pairs;
    out[1] = flips;
    max_dev[0] = worst;
}

/* The same candidate pairs decided by the literal form of Eq. 3 (oracle_pred_paper_form,
 * C2 = (float)(2 cos alpha) from the double angle) against the double-precision Eq. 2:
 * out = {pairs, flips, flips with |D - delta| >= 1e-5 m}, max_dev = the largest |D - delta|
 * over the flips.  Diagnostic only: it shows what the cancellation-free form avoids. */
void oracle_flips_paper_form(int32_t R, int32_t C, const float* range, const double* elev,
                             double az_step, int32_t S, float delta, int32_t wrap, int64_t* out,
                             double* max_dev) {
    float delta2 = oracle_delta2(delta);
    double d64 = (double)delta;
    int64_t pairs = 0, flips = 0, far = 0;
    double worst = 0.0;
    for (int32_t r = 0; r < R; ++r) {
        for (int32_t c = 0; c < C; ++c) {
            float a = range[(int64_t)r * C + c];
            if (!oracle_valid(a)) continue;
            for (int32_t k = 1; k <= S; ++k) {
                for (int vert = 0; vert <= 1; ++vert) {
                    int32_t rr = r, cc = c;
                    double alpha;
                    if (vert) {
                        rr = r + k;
                        if (rr >= R) continue;
                        alpha = fabs(elev[rr] - elev[r]);
                    } else {
                        cc = c + k;
                        if (cc >= C) {
                            if (!wrap) continue;
                            cc = cc % C;
                        }
                        alpha = (double)k * az_step;
                    }
                    float b = range[(int64_t)rr * C + cc];
                    if (!oracle_valid(b)) continue;
                    ++pairs;
                    int f32 = oracle_pred_paper_form(a, b, (float)(2.0 * cos(alpha)), delta2);
                    double da = (double)a, db = (double)b;
                    double sa = sin(alpha / 2.0);
                    double D = sqrt((da - db) * (da - db) + 4.0 * da * db * sa * sa);
                    int f64 = D <= d64 ? 1 : 0;
                    if (f32 != f64) {
                        ++flips;
                        double dev = fabs(D - d64);
                        if (dev >= 1e-5) ++far;
                        if (dev > worst) worst = dev;
                    }
                }
            }
        }
    }
    out[0] = pairs;
    out[1] = flips;
    out[2] = far;
    max_dev[0] = worst;
}

/* ------------------------------------------------------------------------------------ */
/* Spherical projection (§I: "a spherical range image projection of the three-dimensional
 * point cloud ... projected back to the point cloud"; §IV-B: the method relies on a
 * one-to-one matching of points and range-image cells).  The paper gives no formulas;
 * the binning below is this implementation's reading:
 *   column c holds azimuth [c*dphi, (c+1)*dphi), counter-clockwise from +x, full turn;
 *   rows are bounded by the midpoints between adjacent beam elevations (sorted), the
 *   outer rows extending half a spacing beyond their beam;
 *   membership is decided by sign tests of fp32 cross products against fp32 boundary
 *   vectors built in double: s_col(c) = cos(c dphi)*y - sin(c dphi)*x,
 *   s_row(m) = cos(m)*z - sin(m)*rho; a point lies in column c iff s_col(c) >= 0 and
 *   s_col(c+1) < 0, and in the row band of sorted boundaries j, j+1 iff s_row(j) >= 0
 *   and s_row(j+1) < 0.
 * Conflicts: the smallest range wins the pixel, ties to the lower point index. */

/* Boundary tables: colb[2*c], colb[2*c+1] = (float)cos, (float)sin of c*az_step for
 * c = 0..C-1; rowb[2*j], rowb[2*j+1] = (float)cos, (float)sin of sorted boundary j,
 * j = 0..R; sorted_row[j] = row index of the j-th lowest beam.  Returns 0, or -1 when
 * R < 2 or two beams share an elevation. */
int32_t oracle_proj_tables(int32_t R, int32_t C, const double* elev, double az_step,
                           float* colb, float* rowb, int32_t* sorted_row) {
    if (R < 2) return -1;
    for (int32_t c = 0; c < C; ++c) {
        double ang = (double)c * az_step;
        colb[2 * c] = (float)cos(ang);
        colb[2 * c + 1] = (float)sin(ang);
    }
    /* insertion sort of row indices by elevation, ascending */
    for (int32_t r = 0; r < R; ++r) sorted_row[r] = r;
    for (int32_t i = 1; i < R; ++i) {
        int32_t v = sorted_row[i];
        int32_t j = i - 1;
        while (j >= 0 && elev[sorted_row[j]] > elev[v]) {
            sorted_row[j + 1] = sorted_row[j];
            --j;
        }
        sorted_row[j + 1] = v;
    }
    for (int32_t i = 1; i < R; ++i)
        if (!(elev[sorted_row[i]] > elev[sorted_row[i - 1]])) return -1;
    for (int32_t j = 0; j <= R; ++j) {
        double m;
        if (j == 0) {
            double e0 = elev[sorted_row[0]], e1 = elev[sorted_row[1]];
            m = e0 - (e1 - e0) / 2.0;
        } else if (j == R) {
            double e0 = elev[sorted_row[R - 2]], e1 = elev[sorted_row[R - 1]];
            m = e1 + (e1 - e0) / 2.0;
        } else {
            m = (elev[sorted_row[j - 1]] + elev[sorted_row[j]]) / 2.0;
        }
        rowb[2 * j] = (float)cos(m);
        rowb[2 * j + 1] = (float)sin(m);
    }
    return 0;
}

static float s_col(const float* colb, int32_t C, int32_t c, float x, float y) {
    int32_t i = c % C;
    float a = colb[2 * i] * y;
    float b = colb[2 * i + 1] * x;
    return a - b;
}

static float s_row(const float* rowb, int32_t j, float z, float rho) {
    float a = rowb[2 * j] * z;
    float b = rowb[2 * j + 1] * rho;
    return a - b;
}

/* Pixel of one point, or -1; range in *rng.  Column: start from the double-precision
 * azimuth estimate and step to the bin whose sign tests hold.  Row: sign tests over all
 * sorted boundaries, scanned in order. */
static int32_t oracle_point_pixel(int32_t R, int32_t C, double az_step, const float* colb,
                                  const float* rowb, const int32_t* sorted_row, float x, float y,
                                  float z, float* rng) {
    float xx = x * x;
    float yy = y * y;
    float zz = z * z;
    float rho2 = xx + yy;
    float r2 = rho2 + zz;
    float rho = sqrtf(rho2);
    float rg = sqrtf(r2);
    *rng = rg;
    if (!oracle_valid(rg)) return -1;
    if (!(rho > 0.0f)) return -1; /* on the sensor axis: no azimuth */
    /* row: the first sorted boundary strictly above the point */
    if (s_row(rowb, 0, z, rho) < 0.0f) return -1;
    int32_t j = -1;
    for (int32_t b = 1; b <= R; ++b) {
        if (s_row(rowb, b, z, rho) < 0.0f) {
            j = b - 1;
            break;
        }
    }
    if (j < 0) return -1;
    /* column */
    double phi = atan2((double)y, (double)x);
    if (phi < 0.0) phi += 6.283185307179586;
    int32_t c = (int32_t)floor(phi / az_step);
    if (c < 0) c = 0;
    if (c >= C) c = C - 1;
    for (int32_t it = 0; it < 2 * C + 4; ++it) {
        if (s_col(colb, C, c + 1, x, y) >= 0.0f) {
            c = (c + 1) % C;
        } else if (s_col(colb, C, c, x, y) < 0.0f) {
            c = (c + C - 1) % C;
        } else {
            break;
        }
    }
    return sorted_row[j] * C + c;
}

/* Projects n points (xyz, n*3 floats).  range_img (R*C) receives the winning range of
 * each pixel (0 where none); pix (n) the pixel of each point or -1; winner (R*C, may be
 * NULL) the winning point index or -1.  Returns 0, or -1 on bad tables / no memory. */
int32_t oracle_project(int32_t R, int32_t C, const double* elev, double az_step, const float* xyz,
                       int64_t n, float* range_img, int32_t* pix, int32_t* winner) {
    int64_t N = (int64_t)R * C;
    float* colb = (float*)malloc(sizeof(float) * 2 * (size_t)C);
    float* rowb = (float*)malloc(sizeof(float) * 2 * (size_t)(R + 1));
    int32_t* srow = (int32_t*)malloc(sizeof(int32_t) * (size_t)R);
    int64_t* win = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    float* best = (float*)malloc(sizeof(float) * (size_t)(N > 0 ? N : 1));
    int32_t rc = 0;
    if (!colb || !rowb || !srow || !win || !best) { rc = -1; goto done; }
    if (oracle_proj_tables(R, C, elev, az_step, colb, rowb, srow) != 0) { rc = -1; goto done; }
    for (int64_t p = 0; p < N; ++p) { win[p] = -1; best[p] = 0.0f; }
    for (int64_t i = 0; i < n; ++i) {
        float rg;
        int32_t p = oracle_point_pixel(R, C, az_step, colb, rowb, srow, xyz[3 * i],
                                       xyz[3 * i + 1], xyz[3 * i + 2], &rg);
        pix[i] = p;
        if (p < 0) continue;
        /* smallest range wins; points are visited in index order, so a strictly smaller
         * range is needed to replace an earlier winner */
        if (win[p] < 0 || rg < best[p]) {
            win[p] = i;
            best[p] = rg;
        }
    }
    for (int64_t p = 0; p < N; ++p) {
        range_img[p] = win[p] < 0 ? 0.0f : best[p];
        if (winner) winner[p] = (int32_t)win[p];
    }
done:
    free(colb); free(rowb); free(srow); free(win); free(best);
    return rc;
}

/* Labels back onto the points (§I, Fig. 1: every point takes its pixel's instance). */
void oracle_scatter(const int32_t* labels, const int32_t* pix, int64_t n, int32_t* point_labels) {
    for (int64_t i = 0; i < n; ++i) point_labels[i] = pix[i] >= 0 ? labels[pix[i]] : -1;
}

/*
 * Ground extraction (§III-A).  Each reading d2 at (r, c) is compared with the reading d1
 * above it (row r-1, the previous channel; rows are channels from the top), alpha being
 * the angle between the two beams.  Eq. 1 gives the angle beta at the upper point between
 * the ray back to the sensor and the segment to the lower point; its tangent form (Eq. 1
 * simplified) needs sin(alpha) and cos(alpha) as pre-computed constants:
 *     tan(beta) = d2 sin(alpha) / (d1 - d2 cos(alpha)).
 * A horizontal surface gives beta = gamma = the depression angle of the upper beam
 * (-elevation of row r-1); a reading spans a horizontal surface when beta lies within
 * +-theta of gamma (the paper: 10 degrees).  Without the division:
 *     num = d2 * sin_a, den = d1 - d2 * cos_a,
 *     horizontal  <=>  den > 0  and  tan(gamma - theta) * den <= num <= tan(gamma + theta) * den
 * (den <= 0 is beta >= 90 degrees; a bound at or past +-90 degrees is -inf / +inf), every
 * operation one fp32 rounding.  The first channel has no channel above: it takes the
 * decision of the second (the paper extends beta_2 to the first channel).  Both readings
 * must be measurements.
 * Height exception (mount_height > 0): a horizontal reading at height z = d sin(e) (from
 * the sensor) above the line z = rho tan(theta) - mount_height (rho = d cos(e), the line
 * from the wheels rising at the threshold slope) is kept.
 * Tables, double then float, rows r = 1..R-1: sa, ca; tlo, thi; and for every row se, ce.
 * mask[p] = 1 for ground.  theta <= 0: no ground.
 */
static int oracle_horizontal(float d1, float d2, float sa, float ca, float tlo, float thi) {
    if (!oracle_valid(d1) || !oracle_valid(d2)) return 0;
    const float num = d2 * sa;
    const float t = d2 * ca;
    const float den = d1 - t;
    if (!(den > 0.0f)) return 0;
    const float lo = tlo * den;
    const float hi = thi * den;
    return num >= lo && num <= hi;
}

void oracle_ground(int32_t R, int32_t C, const float* range, const double* elev, double theta,
                   double mount_height, uint8_t* mask) {
    memset(mask, 0, (size_t)R * C);
    if (!(theta > 0.0) || R < 2) return;
    const double half_pi = 2.0 * atan(1.0);
    float* sa = (float*)calloc((size_t)R, sizeof(float));
    float* ca = (float*)calloc((size_t)R, sizeof(float));
    float* tlo = (float*)calloc((size_t)R, sizeof(float));
    float* thi = (float*)calloc((size_t)R, sizeof(float));
    float* se = (float*)calloc((size_t)R, sizeof(float));
    float* ce = (float*)calloc((size_t)R, sizeof(float));
    if (!sa || !ca || !tlo || !thi || !se || !ce) goto done;
    for (int32_t r = 0; r < R; ++r) {
        se[r] = (float)sin(elev[r]);
        ce[r] = (float)cos(elev[r]);
        if (r == 0) continue;
        const double alpha = fabs(elev[r - 1] - elev[r]);
        const double gamma = -elev[r - 1];
        sa[r] = (float)sin(alpha);
        ca[r] = (float)cos(alpha);
        tlo[r] = gamma - theta <= -half_pi ? -INFINITY : (float)tan(gamma - theta);
        thi[r] = gamma + theta >= half_pi ? INFINITY : (float)tan(gamma + theta);
    }
    const float tth = (float)tan(theta);
    const float h = (float)mount_height;
    for (int32_t r = 0; r < R; ++r) {
        const int32_t rt = r == 0 ? 1 : r; /* the row whose test decides */
        for (int32_t c = 0; c < C; ++c) {
            const float d = range[(size_t)r * C + c];
            if (!oracle_valid(d)) continue;
            const float d1 = range[(size_t)(rt - 1) * C + c];
            const float d2 = range[(size_t)rt * C + c];
            if (!oracle_horizontal(d1, d2, sa[rt], ca[rt], tlo[rt], thi[rt])) continue;
            if (mount_height > 0.0) {
                const float z = d * se[r];
                const float rho = d * ce[r];
                const float line = rho * tth;
                if (z > line - h) continue; /* above the height line: kept */
            }
            mask[(size_t)r * C + c] = 1;
        }
    }
done:
    free(sa);
    free(ca);
    free(tlo);
    free(thi);
    free(se);
    free(ce);
}


/*
 * Diagonal Map Connections (§III-B-2, "MCs along the main diagonal of the range image").
 * The pair (r, c)-(r+k, c+-k) joins two beams k rows and k columns apart; its alpha is the
 * angle between their rays, so Eq. 3's constant is K = 2 - 2 cos(alpha) = |u1 - u2|^2 for
 * the unit rays u1 = (cos e1, 0, sin e1) and u2 = (cos e2 cos(k step), cos e2 sin(k step),
 * sin e2), e1 = elev[r], e2 = elev[r+k] (the same for +k and -k columns).  Computed in
 * double as that squared distance, rounded once.  Kd[r*S + k-1], 0 when r+k >= R.
 */
void oracle_tables_diag(int32_t R, const double* elev, double az_step, int32_t S, float* Kd) {
    for (int32_t r = 0; r < R; ++r) {
        for (int32_t k = 1; k <= S; ++k) {
            float kd = 0.0f;
            if (r + k < R) {
                const double e1 = elev[r], e2 = elev[r + k], ph = (double)k * az_step;
                const double dx = cos(e1) - cos(e2) * cos(ph);
                const double dy = -cos(e2) * sin(ph);
                const double dz = sin(e1) - sin(e2);
                kd = (float)(dx * dx + dy * dy + dz * dz);
            }
            Kd[r * S + (k - 1)] = kd;
        }
    }
}

/*
 * oracle_label with the diagonal Map Connections as well: breadth-first search in raster
 * order (§III-B-1), the candidate neighbours of (r, c) being (r, c+-k) and (r+-k, c) as in
 * oracle_label, and the four diagonal ones (r+-k, c+-k), k = 1..S (columns mod C with
 * wrap, else inside the frame); a diagonal pair uses Kd of its upper row.
 */
int64_t oracle_label_diag(int32_t R, int32_t C, const float* range, const float* Kv,
                          const float* Kh, const float* Kd, int32_t S, float delta, int32_t wrap,
                          int32_t* labels) {
    int64_t N = (int64_t)R * C;
    float delta2 = oracle_delta2(delta);
    int32_t* queue = (int32_t*)malloc((size_t)(N > 0 ? N : 1) * sizeof(int32_t));
    if (!queue) return -1;
    for (int64_t p = 0; p < N; ++p) labels[p] = -1;
    int64_t ncomp = 0;
    for (int64_t p0 = 0; p0 < N; ++p0) {
        if (labels[p0] != -1 || !oracle_valid(range[p0])) continue;
        ++ncomp;
        int64_t head = 0, tail = 0;
        labels[p0] = (int32_t)p0;
        queue[tail++] = (int32_t)p0;
        while (head < tail) {
            int32_t u = queue[head++];
            int32_t ur = u / C, uc = u % C;
            float a = range[u];
            for (int32_t k = 1; k <= S; ++k) {
                /* dr, dc in {-1, 0, 1} x {-1, 0, 1} without (0, 0): axis and diagonal */
                for (int dr = -1; dr <= 1; ++dr) {
                    for (int dc = -1; dc <= 1; ++dc) {
                        if (dr == 0 && dc == 0) continue;
                        int32_t vr = ur + dr * k;
                        int32_t vc = uc + dc * k;
                        if (vr < 0 || vr >= R) continue;
                        if (vc < 0 || vc >= C) {
                            if (!wrap) continue;
                            vc = ((vc % C) + C) % C;
                        }
                        int32_t v = vr * C + vc;
                        if (labels[v] != -1) continue;
                        float b = range[v];
                        if (!oracle_valid(b)) continue;
                        int32_t top = dr > 0 ? ur : vr;
                        float K = dr == 0 ? Kh[ur * S + k - 1]
                                : dc == 0 ? Kv[top * S + k - 1] : Kd[top * S + k - 1];
                        if (oracle_pred(a, b, K, delta2)) {
                            labels[v] = (int32_t)p0;
                            queue[tail++] = v;
                        }
                    }
                }
            }
        }
    }
    free(queue);
    return ncomp;
}
