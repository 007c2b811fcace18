/*
 * hh_oracle.c -- plain, slow FP64 CPU oracle for handheld-SAR imaging (HHFFBPA).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference that the CUDA path is
 * checked against.  It shares no code, header, table or constant generator with
 * the CUDA library; only tests/, the smoke check and the benchmark's CPU
 * baseline may load it.  Every function cites the passage of the paper
 * ("A Fast and Accurate 3-D Reconstruction Algorithm for Near-Range Microwave
 * Imaging with Handheld Synthetic Aperture Radar") that it follows, and every
 * point where the paper is silent states the reading taken.
 *
 * Conventions (all readings of the paper):
 *   - c = 299 792 458 m/s; k = 2 pi f / c (Sec. II-A).
 *   - Monostatic round trip 2k||p - p'|| (Eq. 1, Eq. bpafreqdomain).
 *   - Complex arrays are interleaved (re, im) doubles.
 *   - Images/voxel lists are float64[n][3] points; the caller orders them.
 *
 * Parity notes: the paper prints no value for these functions to compare against.
 * Each is pinned by something other than itself -- a closed form, an invariant, a
 * special case that reduces to a textbook routine, or brute force on tiny inputs --
 * in the CPU tests; none is "parity unpinned".
 */
#define _POSIX_C_SOURCE 199309L
#include <math.h>
#include <stdint.h>
#include <time.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define HHO_C 299792458.0
#define HHO_PI 3.14159265358979323846

typedef int64_t i64;

static double now_s(void) {
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

/* ------------------------------------------------------------------------ */
/* small complex helpers (explicit, no complex.h)                            */
/* ------------------------------------------------------------------------ */
static inline void cmac(double* acc, double ar, double ai, double br, double bi) {
    acc[0] += ar * br - ai * bi;
    acc[1] += ar * bi + ai * br;
}

/* ------------------------------------------------------------------------ */
/* Range compression, Eq. (eq2_rangecompression), discretised.               */
/* Reading: centred baseband zero-padded IFFT without 1/N scaling:           */
/*   P_i[m] = sum_n s[i,n] exp(+j pi (2n - N_f + 1) m / N_fft)                */
/* i.e. exp(+j 2 (k_n - k_c) m dR) with dR = pi / (N_fft dk).  P is periodic  */
/* in m with period N_fft.  The phase index is reduced exactly in integers.  */
/* ------------------------------------------------------------------------ */
int hho_nfft(int n_f, int os_r) {
    i64 want = (i64)n_f * (i64)os_r;
    int n = 1;
    while (n < want) n <<= 1;
    return n;
}

/* exp(+j pi q / n_fft) for q in [0, 2 n_fft) (tab may be NULL: computed per term) */
static void dft_bin(const double* s_ri, int n_f, int n_fft, i64 m, const double* tab, double out[2]) {
    i64 mm = ((m % n_fft) + n_fft) % n_fft;
    i64 period = 2 * (i64)n_fft;
    double acc[2] = {0.0, 0.0};
    for (int n = 0; n < n_f; ++n) {
        i64 q = ((i64)(2 * n - n_f + 1) * mm) % period;
        if (q < 0) q += period;
        double c, s;
        if (tab) {
            c = tab[2 * q];
            s = tab[2 * q + 1];
        } else {
            double ang = HHO_PI * (double)q / (double)n_fft;
            c = cos(ang);
            s = sin(ang);
        }
        cmac(acc, s_ri[2 * n], s_ri[2 * n + 1], c, s);
    }
    out[0] = acc[0];
    out[1] = acc[1];
}

static double* twiddles(int n_fft) {
    double* t = (double*)malloc(sizeof(double) * 4 * (size_t)n_fft);
    for (i64 q = 0; q < 2 * (i64)n_fft; ++q) {
        double ang = HHO_PI * (double)q / (double)n_fft;
        t[2 * q] = cos(ang);
        t[2 * q + 1] = sin(ang);
    }
    return t;
}

/* Profiles P_i[m] for m = m_lo .. m_lo + n_bins - 1 (mod N_fft), all positions. */
void hho_rc_window(const double* echo_ri, i64 n_pos, int n_f, int n_fft, i64 m_lo, int n_bins,
                   double* prof_ri) {
    double* tab = twiddles(n_fft);
#pragma omp parallel for schedule(static)
    for (i64 i = 0; i < n_pos; ++i)
        for (int j = 0; j < n_bins; ++j)
            dft_bin(echo_ri + 2 * i * n_f, n_f, n_fft, m_lo + j, tab, prof_ri + 2 * (i * n_bins + j));
    free(tab);
}

/* ------------------------------------------------------------------------ */
/* Direct BPA in the frequency domain, Eq. (eq2_bpafreqdomain), discretised  */
/* with unit weights: f(p) = sum_i sum_n s[i,n] exp(+j 2 k_n ||p - p'_i||).   */
/* ------------------------------------------------------------------------ */
void hho_bpa_exact(const double* traj, i64 n_pos, const double* freqs, int n_f, const double* echo_ri,
                   const double* pts, i64 n_pts, double* out_ri) {
    double* k = (double*)malloc(sizeof(double) * n_f);
    for (int n = 0; n < n_f; ++n) k[n] = 2.0 * HHO_PI * freqs[n] / HHO_C;
#pragma omp parallel for schedule(dynamic, 16)
    for (i64 q = 0; q < n_pts; ++q) {
        double acc[2] = {0.0, 0.0};
        for (i64 i = 0; i < n_pos; ++i) {
            double dx = pts[3 * q] - traj[3 * i], dy = pts[3 * q + 1] - traj[3 * i + 1],
                   dz = pts[3 * q + 2] - traj[3 * i + 2];
            double R = sqrt(dx * dx + dy * dy + dz * dz);
            const double* s = echo_ri + 2 * i * n_f;
            for (int n = 0; n < n_f; ++n) {
                double ph = 2.0 * k[n] * R;
                cmac(acc, s[2 * n], s[2 * n + 1], cos(ph), sin(ph));
            }
        }
        out_ri[2 * q] = acc[0];
        out_ri[2 * q + 1] = acc[1];
    }
    free(k);
}

/* ------------------------------------------------------------------------ */
/* Range profiles with a stored window and exact on-demand bins outside it.  */
/* ------------------------------------------------------------------------ */
typedef struct {
    const double* echo_ri; /* [n_pos][n_f] */
    i64 n_pos;
    int n_f, n_fft;
    double* win; /* [n_pos][n_bins] profile window, owned */
    i64 m_lo;
    int n_bins;
    double dR, kc, dk;
} hho_prof;

static void prof_init(hho_prof* P, const double* echo_ri, i64 n_pos, const double* freqs, int n_f, int os_r,
                      double R_lo, double R_hi) {
    P->echo_ri = echo_ri;
    P->n_pos = n_pos;
    P->n_f = n_f;
    P->n_fft = hho_nfft(n_f, os_r);
    double k0 = 2.0 * HHO_PI * freqs[0] / HHO_C, k1 = 2.0 * HHO_PI * freqs[n_f - 1] / HHO_C;
    P->dk = (n_f > 1) ? (k1 - k0) / (n_f - 1) : 1.0;
    P->kc = 0.5 * (k0 + k1);
    P->dR = HHO_PI / ((double)P->n_fft * P->dk);
    if (R_lo < 0) R_lo = 0;
    P->m_lo = (i64)floor(R_lo / P->dR) - 1;
    i64 nb = (i64)ceil(R_hi / P->dR) + 2 - P->m_lo;
    if (nb > P->n_fft) nb = P->n_fft;
    if (nb < 2) nb = 2;
    P->n_bins = (int)nb;
    P->win = (double*)malloc(sizeof(double) * 2 * (size_t)n_pos * (size_t)P->n_bins);
    hho_rc_window(echo_ri, n_pos, n_f, P->n_fft, P->m_lo, P->n_bins, P->win);
}

static void prof_free(hho_prof* P) { free(P->win); }

static inline void prof_get(const hho_prof* P, i64 i, i64 m, double out[2]) {
    i64 j = m - P->m_lo;
    if (j >= 0 && j < P->n_bins) {
        out[0] = P->win[2 * (i * P->n_bins + j)];
        out[1] = P->win[2 * (i * P->n_bins + j) + 1];
    } else {
        dft_bin(P->echo_ri + 2 * i * P->n_f, P->n_f, P->n_fft, m, NULL, out);
    }
}

/* BPA on range-compressed data, Eqs. (eq2_rangecompression)-(eq2_bpatimedomain):   */
/*   f(p) = sum_i exp(+j 2 k_c R) [(1-t) P_i[m0] + t P_i[m0+1]],                     */
/*   mu = R / dR, m0 = floor(mu), t = mu - m0  (linear interpolation: a reading).     */
/* Sums over positions perm[b..e) (or b..e when perm is NULL).                        */
static void bpa_rc_point(const hho_prof* P, const double* traj, const i64* perm, i64 b, i64 e, const double p[3],
                         double out[2]) {
    double acc[2] = {0.0, 0.0};
    for (i64 jj = b; jj < e; ++jj) {
        i64 i = perm ? perm[jj] : jj;
        double dx = p[0] - traj[3 * i], dy = p[1] - traj[3 * i + 1], dz = p[2] - traj[3 * i + 2];
        double R = sqrt(dx * dx + dy * dy + dz * dz);
        double mu = R / P->dR;
        double fl = floor(mu);
        double t = mu - fl;
        i64 m0 = (i64)fl;
        double a0[2], a1[2];
        prof_get(P, i, m0, a0);
        prof_get(P, i, m0 + 1, a1);
        double vr = (1.0 - t) * a0[0] + t * a1[0], vi = (1.0 - t) * a0[1] + t * a1[1];
        double ph = 2.0 * P->kc * R;
        cmac(acc, vr, vi, cos(ph), sin(ph));
    }
    out[0] = acc[0];
    out[1] = acc[1];
}

static void range_bounds(const double* traj, i64 n_pos, const double* pts, i64 n_pts, double* lo, double* hi) {
    /* distance bounds from the bounding boxes of both point sets */
    double bmin[3] = {1e300, 1e300, 1e300}, bmax[3] = {-1e300, -1e300, -1e300};
    double qmin[3] = {1e300, 1e300, 1e300}, qmax[3] = {-1e300, -1e300, -1e300};
    for (i64 i = 0; i < n_pos; ++i)
        for (int d = 0; d < 3; ++d) {
            if (traj[3 * i + d] < bmin[d]) bmin[d] = traj[3 * i + d];
            if (traj[3 * i + d] > bmax[d]) bmax[d] = traj[3 * i + d];
        }
    for (i64 i = 0; i < n_pts; ++i)
        for (int d = 0; d < 3; ++d) {
            if (pts[3 * i + d] < qmin[d]) qmin[d] = pts[3 * i + d];
            if (pts[3 * i + d] > qmax[d]) qmax[d] = pts[3 * i + d];
        }
    double s_lo = 0, s_hi = 0;
    for (int d = 0; d < 3; ++d) {
        double gap = fmax(0.0, fmax(qmin[d] - bmax[d], bmin[d] - qmax[d]));
        double span = fmax(fabs(qmax[d] - bmin[d]), fabs(bmax[d] - qmin[d]));
        s_lo += gap * gap;
        s_hi += span * span;
    }
    *lo = sqrt(s_lo);
    *hi = sqrt(s_hi);
}

/* BPA-RC over all positions at arbitrary points. */
void hho_bpa_rc(const double* traj, i64 n_pos, const double* freqs, int n_f, int os_r, const double* echo_ri,
                const double* pts, i64 n_pts, double* out_ri) {
    double lo, hi;
    range_bounds(traj, n_pos, pts, n_pts, &lo, &hi);
    hho_prof P;
    prof_init(&P, echo_ri, n_pos, freqs, n_f, os_r, lo, hi);
#pragma omp parallel for schedule(dynamic, 16)
    for (i64 q = 0; q < n_pts; ++q) bpa_rc_point(&P, traj, NULL, 0, n_pos, pts + 3 * q, out_ri + 2 * q);
    prof_free(&P);
}

/* Profile parameters as the oracle defines them: out = {n_fft, dR, kc, dk}. */
void hho_rc_params(const double* freqs, int n_f, int os_r, double* out4) {
    int n_fft = hho_nfft(n_f, os_r);
    double k0 = 2.0 * HHO_PI * freqs[0] / HHO_C, k1 = 2.0 * HHO_PI * freqs[n_f - 1] / HHO_C;
    double dk = (n_f > 1) ? (k1 - k0) / (n_f - 1) : 1.0;
    out4[0] = n_fft;
    out4[1] = HHO_PI / ((double)n_fft * dk);
    out4[2] = 0.5 * (k0 + k1);
    out4[3] = dk;
}

/* ------------------------------------------------------------------------ */
/* Spectral design of a subarray, Sec. III.                                   */
/* A subarray is its x'/y' bounds rect = {a = x'min, b = x'max, e = y'min,     */
/* g = y'max}.  Reading: the design plane z' = 0 of the key points is the mean */
/* aperture height zbar, so the design uses zh = z - zbar; Delta x', Delta y'  */
/* in beta, Phi and n are the SUBARRAY extents (the only reading for which the  */
/* boresight condition k7 = k6 holds).                                          */
/* ------------------------------------------------------------------------ */
static inline double clampd(double v, double lo, double hi) {
    /* nearest point of [lo, hi], with the strict tests of the x'_0 definition */
    if (v < lo) return lo;
    if (v > hi) return hi;
    return v;
}

static inline double dist2d(double x, double y, double zh, double X, double Y) {
    return sqrt((x - X) * (x - X) + (y - Y) * (y - Y) + zh * zh);
}

/* k_0(p', p, k) = 2k grad_p ||p - p'|| with p' = (X, Y, zbar), Eq. (eq_kfun_posp). */
static void k0vec(double X, double Y, const double p[3], double zbar, double k, double out[3]) {
    double dx = p[0] - X, dy = p[1] - Y, dz = p[2] - zbar;
    double d = sqrt(dx * dx + dy * dy + dz * dz);
    out[0] = 2 * k * dx / d;
    out[1] = 2 * k * dy / d;
    out[2] = 2 * k * dz / d;
}

/* Key points k1..k7 (Sec. III, key-point definition; Eqs. eq_spv_scl,          */
/* eq_spv_scl_comsol, eq_4r_sum and the boresight choice of beta) and the LLT      */
/* spatial matrix T_s = [v1; v2; v3] / 2 pi (Eq. eq3_lltmatrix).                  */
/* out: k[7][3] then Ts[3][3] (row-major), 30 doubles.                            */
void hho_keypoints(const double rect[4], double zbar, double kmin, double kmax, const double p[3], double* out) {
    double a = rect[0], b = rect[1], e = rect[2], g = rect[3];
    double x0 = clampd(p[0], a, b), y0 = clampd(p[1], e, g);
    double k1[3], k2[3], k3[3], k4[3], k5[3] = {0, 0, 0}, k6[3], k7[3], t[3];
    k0vec(a, y0, p, zbar, kmax, k1);
    k0vec(b, y0, p, zbar, kmax, k2);
    k0vec(x0, e, p, zbar, kmax, k3);
    k0vec(x0, g, p, zbar, kmax, k4);
    double cx[4] = {a, a, b, b}, cy[4] = {e, g, e, g};
    for (int c = 0; c < 4; ++c) {
        k0vec(cx[c], cy[c], p, zbar, kmin, t);
        for (int d = 0; d < 3; ++d) k5[d] += 0.25 * t[d];
    }
    double n5 = sqrt(k5[0] * k5[0] + k5[1] * k5[1] + k5[2] * k5[2]);
    for (int d = 0; d < 3; ++d) k6[d] = 2 * kmax * k5[d] / n5;
    double zh = p[2] - zbar, r = 0;
    for (int c = 0; c < 4; ++c) r += dist2d(p[0], p[1], zh, cx[c], cy[c]);
    double C2 = 4 * (b - a) * (b - a) + 4 * (g - e) * (g - e);
    double beta = kmax * r / (kmin * sqrt(r * r - C2));
    for (int d = 0; d < 3; ++d) k7[d] = beta * k5[d];
    double* o = out;
    const double* ks[7] = {k1, k2, k3, k4, k5, k6, k7};
    for (int i = 0; i < 7; ++i)
        for (int d = 0; d < 3; ++d) *o++ = ks[i][d];
    for (int d = 0; d < 3; ++d) o[d] = (k2[d] - k1[d]) / (2 * HHO_PI);
    for (int d = 0; d < 3; ++d) o[3 + d] = (k4[d] - k3[d]) / (2 * HHO_PI);
    for (int d = 0; d < 3; ++d) o[6 + d] = (k7[d] - k5[d]) / (2 * HHO_PI);
}

/* (u, v, n) coordinates (Eq. eq_uvw_xyz) and the SDC phase Phi (Eq. eq_sdc_phi). */
static void uvn_phi(const double rect[4], double zbar, double kmin, double kmax, const double p[3], double w[4]) {
    double a = rect[0], b = rect[1], e = rect[2], g = rect[3];
    double x = p[0], y = p[1], zh = p[2] - zbar;
    double x0 = clampd(x, a, b), y0 = clampd(y, e, g);
    double u = kmax / HHO_PI * (dist2d(x, y, zh, a, y0) - dist2d(x, y, zh, b, y0));
    double v = kmax / HHO_PI * (dist2d(x, y, zh, x0, e) - dist2d(x, y, zh, x0, g));
    double r = dist2d(x, y, zh, a, e) + dist2d(x, y, zh, a, g) + dist2d(x, y, zh, b, e) + dist2d(x, y, zh, b, g);
    double C2 = 4 * (b - a) * (b - a) + 4 * (g - e) * (g - e);
    double S = sqrt(r * r - C2);
    w[0] = u;
    w[1] = v;
    w[2] = kmax / (4 * HHO_PI) * S - kmin / (4 * HHO_PI) * r;
    w[3] = kmax / 4 * S + kmin / 4 * r;
}

void hho_uvn(const double rect[4], double zbar, double kmin, double kmax, const double* pts, i64 n, double* out4) {
    for (i64 i = 0; i < n; ++i) uvn_phi(rect, zbar, kmin, kmax, pts + 3 * i, out4 + 4 * i);
}

/* Jacobian of (u, v, n): by Eq. (eq_duvw_relp) it is T_s up to the signs of the */
/* printed potentials, which give grad u = -v1/2pi, grad v = -v2/2pi,            */
/* grad n = +v3/2pi.  Built from the key points.                                  */
static void uvn_jacobian(const double rect[4], double zbar, double kmin, double kmax, const double p[3],
                         double J[9]) {
    double kp[30];
    hho_keypoints(rect, zbar, kmin, kmax, p, kp);
    const double* Ts = kp + 21;
    for (int d = 0; d < 3; ++d) {
        J[d] = -Ts[d];
        J[3 + d] = -Ts[3 + d];
        J[6 + d] = Ts[6 + d];
    }
}

static int solve3(const double A[9], const double rhs[3], double x[3]) {
    double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                 A[2] * (A[3] * A[7] - A[4] * A[6]);
    if (!(fabs(det) > 0)) return 0;
    double inv[9];
    inv[0] = (A[4] * A[8] - A[5] * A[7]) / det;
    inv[1] = -(A[1] * A[8] - A[2] * A[7]) / det;
    inv[2] = (A[1] * A[5] - A[2] * A[4]) / det;
    inv[3] = -(A[3] * A[8] - A[5] * A[6]) / det;
    inv[4] = (A[0] * A[8] - A[2] * A[6]) / det;
    inv[5] = -(A[0] * A[5] - A[2] * A[3]) / det;
    inv[6] = (A[3] * A[7] - A[4] * A[6]) / det;
    inv[7] = -(A[0] * A[7] - A[1] * A[6]) / det;
    inv[8] = (A[0] * A[4] - A[1] * A[3]) / det;
    for (int i = 0; i < 3; ++i) x[i] = inv[3 * i] * rhs[0] + inv[3 * i + 1] * rhs[1] + inv[3 * i + 2] * rhs[2];
    return 1;
}

/* ------------------------------------------------------------------------ */
/* Preimage of a (u, v, n) target: the non-uniform xyz sampling point of a   */
/* uniform (u, v, n) grid node (Sec. IV-A: grids "converted to non-uniform   */
/* sampling grids in (x,y,z) through (eq_uvw_xyz)").  The paper gives no     */
/* inverse.  Reading: the unique point with zh > 0 solving uvn(p) = target.  */
/* Every distance of Eq. eq_uvw_xyz depends on zh only through zh^2, so the  */
/* solver works in (x, y, s = zh^2), where the map stays regular at the      */
/* design plane (it folds there in zh) and s < 0 lies beyond the fold: damped */
/* Newton with the analytic Jacobian from the far-field direction-cosine      */
/* estimate, then a homotopy from the subarray boresight as the fallback.     */
/* A point is feasible when the solution has zh >= zh_floor.                  */
/* ------------------------------------------------------------------------ */
static inline double dist_s(double x, double y, double s, double X, double Y) {
    double q = (x - X) * (x - X) + (y - Y) * (y - Y) + s;
    return sqrt(q > 1e-300 ? q : 1e-300);
}

/* (u, v, n) and their derivatives in (x, y, s) */
static void uvn_s(const double rect[4], double kmin, double kmax, double x, double y, double s, double w[3],
                  double* J) {
    double a = rect[0], b = rect[1], e = rect[2], g = rect[3];
    double x0 = clampd(x, a, b), y0 = clampd(y, e, g);
    double da = dist_s(x, y, s, a, y0), db = dist_s(x, y, s, b, y0);
    double de = dist_s(x, y, s, x0, e), dg = dist_s(x, y, s, x0, g);
    double cx[4] = {a, a, b, b}, cy[4] = {e, g, e, g}, d[4], r = 0;
    for (int j = 0; j < 4; ++j) {
        d[j] = dist_s(x, y, s, cx[j], cy[j]);
        r += d[j];
    }
    double C2 = 4 * (b - a) * (b - a) + 4 * (g - e) * (g - e);
    double S = sqrt(r * r - C2 > 0 ? r * r - C2 : 0);
    w[0] = kmax / HHO_PI * (da - db);
    w[1] = kmax / HHO_PI * (de - dg);
    w[2] = kmax / (4 * HHO_PI) * S - kmin / (4 * HHO_PI) * r;
    if (!J) return;
    /* y'_0 and x'_0 are constant where the clamp is active and cancel otherwise */
    J[0] = kmax / HHO_PI * ((x - a) / da - (x - b) / db);
    J[1] = kmax / HHO_PI * ((y - y0) / da - (y - y0) / db);
    J[2] = kmax / HHO_PI * 0.5 * (1 / da - 1 / db);
    J[3] = kmax / HHO_PI * ((x - x0) / de - (x - x0) / dg);
    J[4] = kmax / HHO_PI * ((y - e) / de - (y - g) / dg);
    J[5] = kmax / HHO_PI * 0.5 * (1 / de - 1 / dg);
    double dn = (kmax * r / (S > 1e-300 ? S : 1e-300) - kmin) / (4 * HHO_PI), gx = 0, gy = 0, gs = 0;
    for (int j = 0; j < 4; ++j) {
        gx += (x - cx[j]) / d[j];
        gy += (y - cy[j]) / d[j];
        gs += 0.5 / d[j];
    }
    J[6] = dn * gx;
    J[7] = dn * gy;
    J[8] = dn * gs;
}

static double resid_s(const double rect[4], double kmin, double kmax, const double q[3], const double tgt[3],
                      double res[3]) {
    double w[3];
    uvn_s(rect, kmin, kmax, q[0], q[1], q[2], w, NULL);
    double m = 0;
    for (int d = 0; d < 3; ++d) {
        res[d] = w[d] - tgt[d];
        if (fabs(res[d]) > m) m = fabs(res[d]);
    }
    return m;
}

static int newton_s(const double rect[4], double kmin, double kmax, const double tgt[3], double q[3], int max_it,
                    double tol) {
    double res[3];
    double rn = resid_s(rect, kmin, kmax, q, tgt, res);
    for (int it = 0; it < max_it; ++it) {
        if (rn <= tol) return 1;
        double J[9], st[3], w[3];
        uvn_s(rect, kmin, kmax, q[0], q[1], q[2], w, J);
        if (!solve3(J, res, st)) return 0;
        double lam = 1.0;
        int accepted = 0;
        for (int bt = 0; bt < 40; ++bt) {
            double c[3] = {q[0] - lam * st[0], q[1] - lam * st[1], q[2] - lam * st[2]}, r2[3];
            double rq = resid_s(rect, kmin, kmax, c, tgt, r2);
            if (rq < rn) {
                q[0] = c[0]; q[1] = c[1]; q[2] = c[2];
                rn = rq;
                res[0] = r2[0]; res[1] = r2[1]; res[2] = r2[2];
                accepted = 1;
                break;
            }
            lam *= 0.5;
        }
        if (!accepted) return rn <= tol;
    }
    return rn <= tol;
}

/* returns 1 and p = (x, y, z) when feasible */
static int preimage(const double rect[4], double zbar, double kmin, double kmax, double zh_floor, double zh_mid,
                    const double tgt[3], double p[3]) {
    const double tol = 1e-10;
    double a = rect[0], b = rect[1], e = rect[2], g = rect[3];
    double xc = 0.5 * (a + b), yc = 0.5 * (e + g);
    double usat = kmax / HHO_PI * (b - a), vsat = kmax / HHO_PI * (g - e);
    double sx = tgt[0] / usat, sy = tgt[1] / vsat;
    double s2 = sx * sx + sy * sy;
    if (s2 > 0.98) {
        sx *= sqrt(0.98 / s2);
        sy *= sqrt(0.98 / s2);
        s2 = 0.98;
    }
    /* far-field range from n ~ (kmax-kmin) R / pi - kmax C^2 / (32 pi R) */
    double C2 = 4 * (b - a) * (b - a) + 4 * (g - e) * (g - e);
    double A = (kmax - kmin) / HHO_PI, Bq = kmax * C2 / (32 * HHO_PI);
    double R = (tgt[2] + sqrt(tgt[2] * tgt[2] + 4 * A * Bq)) / (2 * A);
    if (!(R > 1e-4)) R = 1e-4;
    double q[3] = {xc + sx * R, yc + sy * R, R * R * (1 - s2)};
    int ok = newton_s(rect, kmin, kmax, tgt, q, 100, tol);
    if (!ok) {
        /* homotopy from the boresight point at mid depth */
        double w0[3];
        q[0] = xc; q[1] = yc; q[2] = zh_mid * zh_mid;
        uvn_s(rect, kmin, kmax, q[0], q[1], q[2], w0, NULL);
        ok = 1;
        for (int s = 1; s <= 32 && ok; ++s) {
            double lam = s / 32.0;
            double ts[3] = {w0[0] + lam * (tgt[0] - w0[0]), w0[1] + lam * (tgt[1] - w0[1]),
                            w0[2] + lam * (tgt[2] - w0[2])};
            ok = newton_s(rect, kmin, kmax, ts, q, 60, s == 32 ? tol : 1e-7);
        }
    }
    p[0] = q[0];
    p[1] = q[1];
    p[2] = zbar + sqrt(q[2] > 0 ? q[2] : 0);
    if (!ok) return 0;
    return q[2] >= zh_floor * zh_floor;
}

/* Jacobians for tests: the key-point (T_s) Jacobian of (u, v, n) in (x, y, z) and the solver's in (x, y, s). */
void hho_jacobian_ts(const double rect[4], double zbar, double kmin, double kmax, const double p[3], double* J) {
    uvn_jacobian(rect, zbar, kmin, kmax, p, J);
}

void hho_jacobian_s(const double rect[4], double kmin, double kmax, double x, double y, double s, double* J) {
    double w[3];
    uvn_s(rect, kmin, kmax, x, y, s, w, J);
}

/* Batch preimage for tests: ok[i] = 1 when feasible. */
void hho_preimage(const double rect[4], double zbar, double kmin, double kmax, double zh_floor, double zh_mid,
                  const double* tgt, i64 n, double* xyz, int32_t* ok) {
#pragma omp parallel for schedule(dynamic, 64)
    for (i64 i = 0; i < n; ++i) ok[i] = preimage(rect, zbar, kmin, kmax, zh_floor, zh_mid, tgt + 3 * i, xyz + 3 * i);
}

/* ------------------------------------------------------------------------ */
/* Interpolation kernel (the paper does not specify one, Sec. IV-A).         */
/* Reading: the least-squares optimal fractional-delay interpolator for a    */
/* signal whose spectrum fills the unit box after SDC+LLT (Eq.               */
/* eq_llt_spcm_trans: |kappa| <= pi per coordinate), sampled with step 1/eta: */
/* flat spectrum on |f| <= 1/(2 eta) cycles/sample.  Taps at offsets          */
/* o = -(T/2-1) .. T/2 around floor(index); weights h(tau) = G^-1 r(tau) with */
/* G_ij = sinc((o_i - o_j)/eta), r_i = sinc((o_i - tau)/eta).                  */
/* ------------------------------------------------------------------------ */
static double sincpi(double x) {
    if (x == 0.0) return 1.0;
    return sin(HHO_PI * x) / (HHO_PI * x);
}

typedef struct {
    int taps;
    double eta;
    double L[64]; /* Cholesky factor of G, taps <= 8 */
} hho_kernel;

static int kernel_init(hho_kernel* K, int taps, double eta) {
    if (taps < 2 || taps > 8 || (taps & 1)) return 0;
    K->taps = taps;
    K->eta = eta;
    int o0 = -(taps / 2 - 1);
    double G[64];
    for (int i = 0; i < taps; ++i)
        for (int j = 0; j < taps; ++j) G[i * taps + j] = sincpi((double)(i - j) / eta);
    memset(K->L, 0, sizeof(K->L));
    for (int i = 0; i < taps; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = G[i * taps + j];
            for (int k = 0; k < j; ++k) s -= K->L[i * taps + k] * K->L[j * taps + k];
            if (i == j) {
                if (!(s > 0)) return 0;
                K->L[i * taps + i] = sqrt(s);
            } else
                K->L[i * taps + j] = s / K->L[j * taps + j];
        }
    (void)o0;
    return 1;
}

static void kernel_weights(const hho_kernel* K, double tau, double* w) {
    int T = K->taps, o0 = -(T / 2 - 1);
    double r[8], y[8];
    for (int i = 0; i < T; ++i) r[i] = sincpi(((double)(o0 + i) - tau) / K->eta);
    for (int i = 0; i < T; ++i) {
        double s = r[i];
        for (int k = 0; k < i; ++k) s -= K->L[i * T + k] * y[k];
        y[i] = s / K->L[i * T + i];
    }
    for (int i = T - 1; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < T; ++k) s -= K->L[k * T + i] * w[k];
        w[i] = s / K->L[i * T + i];
    }
}

/* weights for a batch of tau values: w[n][taps] */
int hho_ls_weights(int taps, double eta, const double* tau, i64 n, double* w) {
    hho_kernel K;
    if (!kernel_init(&K, taps, eta)) return -1;
    for (i64 i = 0; i < n; ++i) kernel_weights(&K, tau[i], w + i * taps);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Plan: subarray tree and compressed sampling grids (Sec. IV-A).            */
/* ------------------------------------------------------------------------ */
typedef struct {
    int depth;       /* binary depth (0 = root) */
    int level;       /* materialised level: 0 = leaves .. n_levels-1 = root */
    int t;           /* merges above this node (root: 0) */
    i64 begin, end;  /* member range in perm */
    double rect[4];  /* a, b, e, g after the minimum-extent rule */
    double zbar;     /* design plane: mean member height */
    double zmin, zmax; /* member height range */
    double lo[3];    /* lattice origin in (u, v, n) */
    double eta[3];   /* lattice density (samples per unit) per axis */
    i64 N[3];        /* lattice sizes */
    i64 child0, nchild;
} hho_node;

typedef struct {
    i64 n_pos;
    const double* traj; /* caller-owned, [n_pos][3] */
    double kmin, kmax, zbar, zh_floor, zh_mid, min_ext;
    double grid[9]; /* x0 y0 z0 dx dy dz nx ny nz */
    int leaf_size, merge_factor, taps, os_r;
    double eta;
    int depth_leaves, n_levels;
    i64* perm;
    i64 n_nodes;
    hho_node* nodes;    /* grouped by level, leaves first; root last */
    i64* level_start;   /* [n_levels + 1] */
    hho_kernel K;
} hho_plan;

typedef struct {
    double key;
    i64 idx;
} keyed;

static int cmp_keyed(const void* A, const void* B) {
    const keyed* a = (const keyed*)A;
    const keyed* b = (const keyed*)B;
    if (a->key < b->key) return -1;
    if (a->key > b->key) return 1;
    return (a->idx < b->idx) ? -1 : (a->idx > b->idx);
}

/* Spectral extent of a subarray's compressed subimage.  Sec. III bounds the  */
/* local spectrum of the SDC+LLT subimage by the unit box |kappa_d| <= pi      */
/* (Eq. eq_llt_spcm_trans); the paper notes the bound loosens for the last     */
/* levels, where subarrays are large.  Reading: measure it.  For probe points p */
/* of D (corners, face centres, centre) and local spectral components           */
/* K = 2k (p - p')/|p - p'| (Eq. eq_kxyz_posp) with p' on the subarray's border */
/* (4 points per edge) at the lowest and highest member heights -- the paper   */
/* ignores z' fluctuation (Sec. II-B), which small subarrays cannot -- and      */
/* k in {k_min, k_max}, the                                                     */
/* transformed frequency is kappa = J^-T (K - k_c) with J the Jacobian of       */
/* (u, v, n) and k_c = (k5 + k7)/2 = grad Phi (Eq. eq_dp_kc).  rho_d is the     */
/* largest |kappa_d| / pi, rounded up to a multiple of 1/64.                    */
static void spectral_extent(const hho_plan* pl, const double rect[4], double zbar, double zlo, double zhi,
                            double rho[3]) {
    const double* G = pl->grid;
    double xs[3] = {G[0], G[0] + 0.5 * G[3] * (G[6] - 1), G[0] + G[3] * (G[6] - 1)};
    double ys[3] = {G[1], G[1] + 0.5 * G[4] * (G[7] - 1), G[1] + G[4] * (G[7] - 1)};
    double zs[3] = {G[2], G[2] + 0.5 * G[5] * (G[8] - 1), G[2] + G[5] * (G[8] - 1)};
    double a = rect[0], b = rect[1], e = rect[2], g = rect[3];
    double bx[12], by[12];
    for (int q = 0; q < 4; ++q) {
        double s = q / 4.0;
        bx[q] = a + s * (b - a); by[q] = e;           /* bottom edge */
        bx[4 + q] = b; by[4 + q] = e + s * (g - e);   /* right edge */
        bx[8 + q] = b - s * (b - a); by[8 + q] = g;   /* top edge */
    }
    double ex[16], ey[16];
    for (int q = 0; q < 12; ++q) { ex[q] = bx[q]; ey[q] = by[q]; }
    for (int q = 0; q < 4; ++q) { ex[12 + q] = a; ey[12 + q] = g - (q / 4.0) * (g - e); } /* left edge */
    rho[0] = rho[1] = rho[2] = 1.0;
    for (int ix = 0; ix < 3; ++ix)
        for (int iy = 0; iy < 3; ++iy)
            for (int iz = 0; iz < 3; ++iz) {
                int mids = (ix == 1) + (iy == 1) + (iz == 1);
                if (mids == 1) continue; /* corners (0), face centres (2), centre (3) */
                double p[3] = {xs[ix], ys[iy], zs[iz]};
                double kp[30];
                hho_keypoints(rect, zbar, pl->kmin, pl->kmax, p, kp);
                double kc[3], J[9];
                for (int d = 0; d < 3; ++d) kc[d] = 0.5 * (kp[12 + d] + kp[18 + d]);
                const double* Ts = kp + 21;
                for (int d = 0; d < 3; ++d) { J[d] = -Ts[d]; J[3 + d] = -Ts[3 + d]; J[6 + d] = Ts[6 + d]; }
                /* kappa solves J^T kappa = K - k_c */
                double JT[9] = {J[0], J[3], J[6], J[1], J[4], J[7], J[2], J[5], J[8]};
                for (int q = 0; q < 16; ++q)
                    for (int kk = 0; kk < 4; ++kk) {
                        double K[3];
                        k0vec(ex[q], ey[q], p, (kk & 2) ? zhi : zlo, (kk & 1) ? pl->kmax : pl->kmin, K);
                        double rhs[3] = {K[0] - kc[0], K[1] - kc[1], K[2] - kc[2]}, kap[3];
                        if (!solve3(JT, rhs, kap)) continue;
                        for (int d = 0; d < 3; ++d) {
                            double r = fabs(kap[d]) / HHO_PI;
                            if (r > rho[d]) rho[d] = r;
                        }
                    }
            }
    for (int d = 0; d < 3; ++d) rho[d] = ceil(rho[d] * 64.0) / 64.0;
}

/* Extremes of (u, v, n) over the box D.  Reading (the paper gives no rule):   */
/* u grows with x and is monotone in h^2 = (y - y'_0)^2 + zh^2 on an x-face, so */
/* its extremes lie on the x faces at y in {y_lo, y_hi, clamp(e), clamp(g)} and */
/* z in {z_lo, z_hi}; likewise v.  n grows with zh and with r, and r is least   */
/* at the clamped subarray centre and greatest at a box corner.                 */
static void lattice_bbox(const hho_plan* pl, const double rect[4], double zbar, double mn[3], double mx[3]) {
    const double* G = pl->grid;
    double xl = G[0], xh = G[0] + G[3] * (G[6] - 1), yl = G[1], yh = G[1] + G[4] * (G[7] - 1), zl = G[2],
           zhh = G[2] + G[5] * (G[8] - 1);
    double a = rect[0], b = rect[1], e = rect[2], g = rect[3];
    double yc[4] = {yl, yh, clampd(e, yl, yh), clampd(g, yl, yh)};
    double xcnd[4] = {xl, xh, clampd(a, xl, xh), clampd(b, xl, xh)};
    double zc[2] = {zl, zhh};
    double w[4], p[3];
    mn[0] = mn[1] = mn[2] = 1e300;
    mx[0] = mx[1] = mx[2] = -1e300;
    for (int i = 0; i < 4; ++i)
        for (int k = 0; k < 2; ++k) {
            p[0] = xl; p[1] = yc[i]; p[2] = zc[k];
            uvn_phi(rect, zbar, pl->kmin, pl->kmax, p, w);
            if (w[0] < mn[0]) mn[0] = w[0];
            p[0] = xh;
            uvn_phi(rect, zbar, pl->kmin, pl->kmax, p, w);
            if (w[0] > mx[0]) mx[0] = w[0];
            p[0] = xcnd[i]; p[1] = yl;
            uvn_phi(rect, zbar, pl->kmin, pl->kmax, p, w);
            if (w[1] < mn[1]) mn[1] = w[1];
            p[1] = yh;
            uvn_phi(rect, zbar, pl->kmin, pl->kmax, p, w);
            if (w[1] > mx[1]) mx[1] = w[1];
        }
    p[0] = clampd(0.5 * (a + b), xl, xh);
    p[1] = clampd(0.5 * (e + g), yl, yh);
    p[2] = zl;
    uvn_phi(rect, zbar, pl->kmin, pl->kmax, p, w);
    mn[2] = w[2];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            p[0] = i ? xh : xl; p[1] = j ? yh : yl; p[2] = zhh;
            uvn_phi(rect, zbar, pl->kmin, pl->kmax, p, w);
            if (w[2] > mx[2]) mx[2] = w[2];
        }
}

/* Padding (lattice steps beyond D's image) for a node with t merges above it. */
/* Reading: the footprint reaches m = taps/2 steps past a needed point, and the */
/* needed region of a child is its parent's needed region mapped down plus m.   */
/* With 4-way merges the u, v steps double per level down, so their padding     */
/* converges to 2m; n's step does not change, so its padding grows by m per     */
/* level.  One extra step of margin.                                            */
static void node_padding(const hho_plan* pl, int t, i64 pad[3]) {
    i64 m = pl->taps / 2;
    i64 pn = m * t + 1;
    i64 puv = (pl->merge_factor == 4) ? ((m * t < 2 * m ? m * t : 2 * m) + 1) : pn;
    pad[0] = puv;
    pad[1] = puv;
    pad[2] = pn;
}

void hho_plan_destroy(hho_plan* pl) {
    if (!pl) return;
    free(pl->perm);
    free(pl->nodes);
    free(pl->level_start);
    free(pl);
}

/* grid: x0 y0 z0 dx dy dz nx ny nz.  Returns NULL on bad arguments. */
hho_plan* hho_plan_create(const double* traj, i64 n_pos, const double* freqs, int n_f, const double* grid,
                          int leaf_size, int merge_factor, double eta, int taps, int os_r) {
    if (n_pos < 1 || n_f < 2 || leaf_size < 1 || (merge_factor != 2 && merge_factor != 4) || !(eta >= 1.0))
        return NULL;
    hho_plan* pl = (hho_plan*)calloc(1, sizeof(hho_plan));
    pl->n_pos = n_pos;
    pl->traj = traj;
    memcpy(pl->grid, grid, sizeof(pl->grid));
    pl->leaf_size = leaf_size;
    pl->merge_factor = merge_factor;
    pl->eta = eta;
    pl->taps = taps;
    pl->os_r = os_r;
    if (!kernel_init(&pl->K, taps, eta)) {
        free(pl);
        return NULL;
    }
    pl->kmin = 2 * HHO_PI * freqs[0] / HHO_C;
    pl->kmax = 2 * HHO_PI * freqs[n_f - 1] / HHO_C;
    double zs = 0, ztop = -1e300;
    for (i64 i = 0; i < n_pos; ++i) {
        zs += traj[3 * i + 2];
        if (traj[3 * i + 2] > ztop) ztop = traj[3 * i + 2];
    }
    pl->zbar = zs / (double)n_pos;
    /* D must lie in front of every position; a sample point is feasible when  */
    /* it lies at least zh_floor above its subarray's design plane (reading).   */
    double zlo = grid[2] - ztop, zhi = grid[2] + grid[5] * (grid[8] - 1) - pl->zbar;
    if (!(zlo > 0)) {
        free(pl);
        return NULL;
    }
    pl->zh_floor = 0.1 * zlo;
    pl->zh_mid = 0.5 * (grid[2] - pl->zbar + zhi);
    /* minimum subarray extent (reading): half the shortest wavelength */
    pl->min_ext = 0.5 * HHO_C / freqs[n_f - 1];

    /* binary k-d tree: depth d splits along x (d even) or y (d odd) by      */
    /* (coordinate, index) order; the lower half gets floor(n/2) members.    */
    int D = 0;
    while (((i64)1 << (D + 1)) * (i64)leaf_size <= n_pos) ++D;
    pl->depth_leaves = D;
    pl->perm = (i64*)malloc(sizeof(i64) * n_pos);
    for (i64 i = 0; i < n_pos; ++i) pl->perm[i] = i;
    i64* bounds = (i64*)malloc(sizeof(i64) * (((size_t)1 << D) + 1));
    i64* nb = (i64*)malloc(sizeof(i64) * (((size_t)1 << D) + 1));
    i64** all_bounds = (i64**)malloc(sizeof(i64*) * (D + 1));
    bounds[0] = 0;
    bounds[1] = n_pos;
    keyed* tmp = (keyed*)malloc(sizeof(keyed) * n_pos);
    all_bounds[0] = (i64*)malloc(sizeof(i64) * 2);
    memcpy(all_bounds[0], bounds, sizeof(i64) * 2);
    for (int d = 0; d < D; ++d) {
        i64 cnt = (i64)1 << d;
        int axis = d & 1;
        for (i64 j = 0; j < cnt; ++j) {
            i64 b0 = bounds[j], b1 = bounds[j + 1], n = b1 - b0;
            for (i64 q = 0; q < n; ++q) {
                tmp[q].idx = pl->perm[b0 + q];
                tmp[q].key = traj[3 * tmp[q].idx + axis];
            }
            qsort(tmp, (size_t)n, sizeof(keyed), cmp_keyed);
            for (i64 q = 0; q < n; ++q) pl->perm[b0 + q] = tmp[q].idx;
            nb[2 * j] = b0;
            nb[2 * j + 1] = b0 + n / 2;
        }
        nb[2 * cnt] = n_pos;
        memcpy(bounds, nb, sizeof(i64) * (2 * cnt + 1));
        all_bounds[d + 1] = (i64*)malloc(sizeof(i64) * (2 * cnt + 1));
        memcpy(all_bounds[d + 1], bounds, sizeof(i64) * (2 * cnt + 1));
    }
    free(tmp);

    /* materialised depths: D, D - s, D - 2s, ... (> 0), then 0 (the root).   */
    int s = merge_factor == 4 ? 2 : 1;
    int depths[128], nl = 0;
    for (int d = D; d > 0; d -= s) depths[nl++] = d;
    depths[nl++] = 0;
    pl->n_levels = nl;
    pl->level_start = (i64*)malloc(sizeof(i64) * (nl + 1));
    i64 total = 0;
    for (int l = 0; l < nl; ++l) total += (i64)1 << depths[l];
    pl->n_nodes = total;
    pl->nodes = (hho_node*)calloc((size_t)total, sizeof(hho_node));
    i64 at = 0;
    for (int l = 0; l < nl; ++l) {
        pl->level_start[l] = at;
        int d = depths[l];
        i64 cnt = (i64)1 << d;
        for (i64 j = 0; j < cnt; ++j) {
            hho_node* nd = &pl->nodes[at + j];
            nd->depth = d;
            nd->level = l;
            nd->t = nl - 1 - l;
            nd->begin = all_bounds[d][j];
            nd->end = all_bounds[d][j + 1];
            if (l > 0) {
                i64 f = (i64)1 << (depths[l - 1] - d);
                nd->child0 = pl->level_start[l - 1] + j * f;
                nd->nchild = f;
            }
            double a = 1e300, b = -1e300, e = 1e300, g = -1e300, zsum = 0;
            nd->zmin = 1e300;
            nd->zmax = -1e300;
            for (i64 q = nd->begin; q < nd->end; ++q) {
                const double* pp = traj + 3 * pl->perm[q];
                if (pp[0] < a) a = pp[0];
                if (pp[0] > b) b = pp[0];
                if (pp[1] < e) e = pp[1];
                if (pp[1] > g) g = pp[1];
                if (pp[2] < nd->zmin) nd->zmin = pp[2];
                if (pp[2] > nd->zmax) nd->zmax = pp[2];
            }
            /* design plane of the subarray (reading): its members' mean height, */
            /* summed in original index order                                      */
            {
                i64 cnt = nd->end - nd->begin;
                i64* ids = (i64*)malloc(sizeof(i64) * cnt);
                memcpy(ids, pl->perm + nd->begin, sizeof(i64) * cnt);
                for (i64 q = 1; q < cnt; ++q) { /* insertion sort: small ranges are typical */
                    i64 v = ids[q], r = q - 1;
                    while (r >= 0 && ids[r] > v) { ids[r + 1] = ids[r]; --r; }
                    ids[r + 1] = v;
                }
                for (i64 q = 0; q < cnt; ++q) zsum += traj[3 * ids[q] + 2];
                free(ids);
                nd->zbar = zsum / (double)cnt;
            }
            if (b - a < pl->min_ext) {
                double c = 0.5 * (a + b);
                a = c - 0.5 * pl->min_ext;
                b = c + 0.5 * pl->min_ext;
            }
            if (g - e < pl->min_ext) {
                double c = 0.5 * (e + g);
                e = c - 0.5 * pl->min_ext;
                g = c + 0.5 * pl->min_ext;
            }
            nd->rect[0] = a; nd->rect[1] = b; nd->rect[2] = e; nd->rect[3] = g;
            if (l < nl - 1) {
                double mn[3], mx[3], rho[3];
                i64 pad[3];
                lattice_bbox(pl, nd->rect, nd->zbar, mn, mx);
                node_padding(pl, nd->t, pad);
                spectral_extent(pl, nd->rect, nd->zbar, nd->zmin, nd->zmax, rho);
                for (int k = 0; k < 3; ++k) {
                    nd->eta[k] = eta * rho[k];
                    nd->lo[k] = mn[k] - (double)pad[k] / nd->eta[k];
                    nd->N[k] = (i64)ceil((mx[k] - mn[k]) * nd->eta[k]) + 1 + 2 * pad[k];
                }
            }
        }
        at += cnt;
    }
    pl->level_start[nl] = at;
    for (int d = 0; d <= D; ++d) free(all_bounds[d]);
    free(all_bounds);
    free(bounds);
    free(nb);
    return pl;
}

/* Plan summary: {n_levels, n_nodes, depth_leaves}, and per-level node counts. */
void hho_plan_info(const hho_plan* pl, i64* out) {
    out[0] = pl->n_levels;
    out[1] = pl->n_nodes;
    out[2] = pl->depth_leaves;
    for (int l = 0; l <= pl->n_levels; ++l) out[3 + l] = pl->level_start[l];
}

/* Export: perm[n_pos]; per node {level, depth, t, begin, end, child0, nchild, N0, N1, N2}
 * (int64 x 10) and {a, b, e, g, lo0, lo1, lo2, eta0, eta1, eta2, zbar} (double x 11); scalars {zbar, kmin, kmax,
 * zh_floor, zh_mid, min_ext}. */
void hho_plan_export(const hho_plan* pl, i64* perm, i64* nodes_i, double* nodes_d, double* scal) {
    memcpy(perm, pl->perm, sizeof(i64) * pl->n_pos);
    for (i64 k = 0; k < pl->n_nodes; ++k) {
        const hho_node* nd = &pl->nodes[k];
        i64* I = nodes_i + 10 * k;
        I[0] = nd->level; I[1] = nd->depth; I[2] = nd->t; I[3] = nd->begin; I[4] = nd->end;
        I[5] = nd->child0; I[6] = nd->nchild; I[7] = nd->N[0]; I[8] = nd->N[1]; I[9] = nd->N[2];
        double* F = nodes_d + 11 * k;
        for (int q = 0; q < 4; ++q) F[q] = nd->rect[q];
        for (int q = 0; q < 3; ++q) F[4 + q] = nd->lo[q];
        for (int q = 0; q < 3; ++q) F[7 + q] = nd->eta[q];
        F[10] = nd->zbar;
    }
    scal[0] = pl->zbar; scal[1] = pl->kmin; scal[2] = pl->kmax;
    scal[3] = pl->zh_floor; scal[4] = pl->zh_mid; scal[5] = pl->min_ext;
}

/* ------------------------------------------------------------------------ */
/* HHFFBPA evaluation (Sec. IV-A and the merge recursion of Sec. III):        */
/*   leaves:  g_L(q) = exp(-j Phi_L(p_q)) * BPA-RC over L's members at p_q      */
/*   merges:  g_P(q) = exp(-j Phi_P(p_q)) * sum_c f_c(p_q)                       */
/*   final:   f(p)   = sum_{c of root} f_c(p) on the Cartesian voxels            */
/* with f_c(p) = exp(+j Phi_c(p)) * I_c(p), I_c the separable interpolation of   */
/* g_c at lattice index ((u_c(p) - lo) eta, ...).  Reading: when the footprint   */
/* of I_c at p leaves c's lattice or meets an infeasible sample, f_c(p) is the   */
/* BPA-RC of c's members at p (exact fallback).                                  */
/* Only samples needed by the requested output points are computed (demand-     */
/* driven); a sample's value does not depend on which other samples exist.        */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint8_t* need;   /* per lattice point */
    double* val;     /* [N][2] (NaN = missing/infeasible), allocated in the up pass */
} node_data;

static inline i64 lat_index(const hho_node* nd, i64 iu, i64 iv, i64 in) {
    return (iu * nd->N[1] + iv) * nd->N[2] + in;
}

static void lattice_target(const hho_plan* pl, const hho_node* nd, i64 lin, double tgt[3]) {
    i64 in = lin % nd->N[2];
    i64 iv = (lin / nd->N[2]) % nd->N[1];
    i64 iu = lin / (nd->N[2] * nd->N[1]);
    tgt[0] = nd->lo[0] + (double)iu / nd->eta[0];
    tgt[1] = nd->lo[1] + (double)iv / nd->eta[1];
    tgt[2] = nd->lo[2] + (double)in / nd->eta[2];
}

/* footprint of node c at point p: base indices and weights; returns 1 if inside */
typedef struct {
    i64 base[3];
    double w[3][8];
    int inside;
    double phi;
} footprint;

static void make_footprint(const hho_plan* pl, const hho_node* c, const double p[3], footprint* F) {
    double w4[4];
    uvn_phi(c->rect, c->zbar, pl->kmin, pl->kmax, p, w4);
    F->phi = w4[3];
    int T = pl->taps, o0 = -(T / 2 - 1);
    F->inside = 1;
    for (int k = 0; k < 3; ++k) {
        double f = (w4[k] - c->lo[k]) * c->eta[k];
        double fl = floor(f);
        F->base[k] = (i64)fl + o0;
        kernel_weights(&pl->K, f - fl, F->w[k]);
        if (F->base[k] < 0 || F->base[k] + T - 1 > c->N[k] - 1) F->inside = 0;
    }
}

static void mark_footprint(const hho_plan* pl, const hho_node* c, node_data* cd, const footprint* F) {
    int T = pl->taps;
    for (int a = 0; a < T; ++a) {
        i64 iu = F->base[0] + a;
        if (iu < 0 || iu >= c->N[0]) continue;
        for (int b = 0; b < T; ++b) {
            i64 iv = F->base[1] + b;
            if (iv < 0 || iv >= c->N[1]) continue;
            for (int q = 0; q < T; ++q) {
                i64 in = F->base[2] + q;
                if (in < 0 || in >= c->N[2]) continue;
                i64 li = lat_index(c, iu, iv, in);
#pragma omp atomic write
                cd->need[li] = 1;
            }
        }
    }
}

/* returns 1 with out = I_c(p) when the footprint is complete */
static int interp_footprint(const hho_plan* pl, const hho_node* c, const node_data* cd, const footprint* F,
                            double out[2]) {
    if (!F->inside) return 0;
    int T = pl->taps;
    double acc[2] = {0, 0};
    for (int a = 0; a < T; ++a)
        for (int b = 0; b < T; ++b) {
            double wab = F->w[0][a] * F->w[1][b];
            for (int q = 0; q < T; ++q) {
                i64 li = lat_index(c, F->base[0] + a, F->base[1] + b, F->base[2] + q);
                double vr = cd->val[2 * li], vi = cd->val[2 * li + 1];
                if (isnan(vr)) return 0;
                double ww = wab * F->w[2][q];
                acc[0] += ww * vr;
                acc[1] += ww * vi;
            }
        }
    out[0] = acc[0];
    out[1] = acc[1];
    return 1;
}

/* contribution f_c(p) of child c at point p (interpolated or fallback). */
static void child_contrib(const hho_plan* pl, const hho_prof* P, const hho_node* c, const node_data* cd,
                          const double p[3], double out[2], i64* n_fallback) {
    footprint F;
    make_footprint(pl, c, p, &F);
    double I[2];
    if (interp_footprint(pl, c, cd, &F, I)) {
        double cr = cos(F.phi), ci = sin(F.phi);
        out[0] = I[0] * cr - I[1] * ci;
        out[1] = I[0] * ci + I[1] * cr;
    } else {
        bpa_rc_point(P, pl->traj, pl->perm, c->begin, c->end, p, out);
#pragma omp atomic
        (*n_fallback)++;
    }
}

/* stats out (int64[80]): {fallbacks, infeasible needed samples, needed samples, leaf BPA updates,
 * t_profiles, t_topdown, t_leaves, t_final (ns), per-level time ns [8..40), per-level needed [40..72)} */
int hho_hhffbpa(const hho_plan* pl, const double* freqs, int n_f, const double* echo_ri, const double* pts,
                i64 n_pts, double* out_ri, i64* stats) {
    int nl = pl->n_levels;
    const hho_node* root = &pl->nodes[pl->level_start[nl - 1]];
    i64 n_fallback = 0, n_infeasible = 0, n_needed = 0, n_updates = 0;
    i64 lvl_ns[32] = {0}, lvl_need[32] = {0};
    double t0 = now_s();
    /* profiles: window over all positions covering the output points +/- 0.3 m */
    double lo, hi;
    range_bounds(pl->traj, pl->n_pos, pts, n_pts, &lo, &hi);
    hho_prof P;
    prof_init(&P, echo_ri, pl->n_pos, freqs, n_f, pl->os_r, lo - 0.3, hi + 0.3);
    double t_prof = now_s() - t0;

    if (nl == 1) { /* no factorisation: M = 1, plain BPA-RC on the grid */
#pragma omp parallel for schedule(dynamic, 16)
        for (i64 q = 0; q < n_pts; ++q) bpa_rc_point(&P, pl->traj, pl->perm, 0, pl->n_pos, pts + 3 * q, out_ri + 2 * q);
        prof_free(&P);
        if (stats) {
            memset(stats, 0, sizeof(i64) * 80);
            stats[3] = pl->n_pos * n_pts;
            stats[4] = (i64)(1e9 * t_prof);
            stats[7] = (i64)(1e9 * (now_s() - t0 - t_prof));
        }
        return 0;
    }

    node_data* D = (node_data*)calloc((size_t)pl->n_nodes, sizeof(node_data));
    for (i64 k = 0; k < pl->level_start[nl - 1]; ++k) {
        const hho_node* nd = &pl->nodes[k];
        D[k].need = (uint8_t*)calloc((size_t)(nd->N[0] * nd->N[1] * nd->N[2]), 1);
    }
    if (getenv("HHO_MARK_ALL")) /* diagnostic: evaluate every lattice point */
        for (i64 k = 0; k < pl->level_start[nl - 1]; ++k) {
            const hho_node* nd = &pl->nodes[k];
            memset(D[k].need, 1, (size_t)(nd->N[0] * nd->N[1] * nd->N[2]));
        }
    double t1 = now_s();
    /* top-down: mark what the output points need in the root's children */
    for (i64 c = 0; c < root->nchild; ++c) {
        const hho_node* cn = &pl->nodes[root->child0 + c];
#pragma omp parallel for schedule(dynamic, 64)
        for (i64 q = 0; q < n_pts; ++q) {
            footprint F;
            make_footprint(pl, cn, pts + 3 * q, &F);
            mark_footprint(pl, cn, &D[root->child0 + c], &F);
        }
    }
    /* ... and level by level down to the leaves' parents */
    for (int l = nl - 2; l >= 1; --l) {
        for (i64 k = pl->level_start[l]; k < pl->level_start[l + 1]; ++k) {
            const hho_node* nd = &pl->nodes[k];
            i64 NN = nd->N[0] * nd->N[1] * nd->N[2];
#pragma omp parallel for schedule(dynamic, 64)
            for (i64 li = 0; li < NN; ++li) {
                if (!D[k].need[li]) continue;
                double tgt[3], p[3];
                lattice_target(pl, nd, li, tgt);
                if (!preimage(nd->rect, nd->zbar, pl->kmin, pl->kmax, pl->zh_floor, pl->zh_mid, tgt, p)) continue;
                for (i64 c = 0; c < nd->nchild; ++c) {
                    footprint F;
                    make_footprint(pl, &pl->nodes[nd->child0 + c], p, &F);
                    mark_footprint(pl, &pl->nodes[nd->child0 + c], &D[nd->child0 + c], &F);
                }
            }
        }
    }
    double t_top = now_s() - t1;
    /* bottom-up values */
    for (int l = 0; l <= nl - 2; ++l) {
        double tl0 = now_s();
        for (i64 k = pl->level_start[l]; k < pl->level_start[l + 1]; ++k) {
            const hho_node* nd = &pl->nodes[k];
            i64 NN = nd->N[0] * nd->N[1] * nd->N[2];
            D[k].val = (double*)malloc(sizeof(double) * 2 * (size_t)NN);
            i64 loc_need = 0, loc_inf = 0, loc_upd = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : loc_need, loc_inf, loc_upd)
            for (i64 li = 0; li < NN; ++li) {
                double* o = D[k].val + 2 * li;
                o[0] = o[1] = NAN;
                if (!D[k].need[li]) continue;
                ++loc_need;
                double tgt[3], p[3];
                lattice_target(pl, nd, li, tgt);
                if (!preimage(nd->rect, nd->zbar, pl->kmin, pl->kmax, pl->zh_floor, pl->zh_mid, tgt, p)) {
                    ++loc_inf;
                    continue;
                }
                double w4[4];
                uvn_phi(nd->rect, nd->zbar, pl->kmin, pl->kmax, p, w4);
                double f[2] = {0, 0};
                if (l == 0) {
                    bpa_rc_point(&P, pl->traj, pl->perm, nd->begin, nd->end, p, f);
                    loc_upd += nd->end - nd->begin;
                } else {
                    for (i64 c = 0; c < nd->nchild; ++c) {
                        double fc[2];
                        child_contrib(pl, &P, &pl->nodes[nd->child0 + c], &D[nd->child0 + c], p, fc, &n_fallback);
                        f[0] += fc[0];
                        f[1] += fc[1];
                    }
                }
                double cr = cos(w4[3]), ci = -sin(w4[3]);
                o[0] = f[0] * cr - f[1] * ci;
                o[1] = f[0] * ci + f[1] * cr;
            }
            n_needed += loc_need;
            n_infeasible += loc_inf;
            n_updates += loc_upd;
            lvl_need[l] += loc_need;
        }
        lvl_ns[l] = (i64)(1e9 * (now_s() - tl0));
        if (l > 0)
            for (i64 k = pl->level_start[l - 1]; k < pl->level_start[l]; ++k) {
                free(D[k].val);
                D[k].val = NULL;
            }
    }
    double tf0 = now_s();
    /* final: Cartesian voxels */
#pragma omp parallel for schedule(dynamic, 64)
    for (i64 q = 0; q < n_pts; ++q) {
        double f[2] = {0, 0};
        for (i64 c = 0; c < root->nchild; ++c) {
            double fc[2];
            child_contrib(pl, &P, &pl->nodes[root->child0 + c], &D[root->child0 + c], pts + 3 * q, fc, &n_fallback);
            f[0] += fc[0];
            f[1] += fc[1];
        }
        out_ri[2 * q] = f[0];
        out_ri[2 * q + 1] = f[1];
    }
    for (i64 k = 0; k < pl->n_nodes; ++k) {
        free(D[k].need);
        free(D[k].val);
    }
    free(D);
    prof_free(&P);
    if (stats) {
        memset(stats, 0, sizeof(i64) * 80);
        stats[0] = n_fallback;
        stats[1] = n_infeasible;
        stats[2] = n_needed;
        stats[3] = n_updates;
        stats[4] = (i64)(1e9 * t_prof);
        stats[5] = (i64)(1e9 * t_top);
        stats[6] = lvl_ns[0];
        stats[7] = (i64)(1e9 * (now_s() - tf0));
        for (int l = 0; l < nl && l < 32; ++l) {
            stats[8 + l] = lvl_ns[l];
            stats[40 + l] = lvl_need[l];
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Adjoint of the HHFFBPA map (echo -> image values at the points), the      */
/* conjugate transpose of hho_hhffbpa taken step by step in reverse order:    */
/*   final:   x_q -> each root child c: w e^{-j phi_c} x_q into c's footprint */
/*            samples, or (fallback) the BPA-RC adjoint over c's members;     */
/*   merges:  y = e^{+j Phi_P(p)} adj_P[q] -> the same child step at p;       */
/*   leaves:  y = e^{+j Phi_L(p)} adj_L[q] -> BPA-RC adjoint over L's members */
/*            at p: bins m0, m0+1 of each member get (1-t, t) e^{-j 2 k_c R} y;*/
/*   range compression: s[i,n] = sum_m e^{-j theta_n (m mod N)} B_i[m].       */
/* The interpolation/fallback choice depends on geometry alone (footprint    */
/* inside the lattice, every footprint sample feasible), so the forward map  */
/* is linear in the echo and this is its exact adjoint.                       */
/* ------------------------------------------------------------------------ */
typedef struct {
    i64 n_pos, m_lo;
    int n_bins, n_f, n_fft;
    double dR, kc;
    double* win;   /* [n_pos][n_bins][2]: adjoint of the profile window's bins */
    double* extra; /* [n_pos][n_f][2]: bins outside the window, transformed at once */
    /* position-gradient mode (win and extra unused): the forward profiles and the output */
    const hho_prof* P;
    double* grad;  /* [n_pos][3] */
} adj_prof;

static void adj_add_bin(adj_prof* A, i64 i, i64 m, double vr, double vi) {
    i64 j = m - A->m_lo;
    if (j >= 0 && j < A->n_bins) {
        double* w = A->win + 2 * (i * A->n_bins + j);
#pragma omp atomic
        w[0] += vr;
#pragma omp atomic
        w[1] += vi;
        return;
    }
    /* the adjoint of dft_bin for this one bin: conj(e^{+j pi (2n - N_f + 1) (m mod N) / N}) */
    i64 mm = ((m % A->n_fft) + A->n_fft) % A->n_fft, period = 2 * (i64)A->n_fft;
    for (int n = 0; n < A->n_f; ++n) {
        i64 q = ((i64)(2 * n - A->n_f + 1) * mm) % period;
        if (q < 0) q += period;
        double ang = HHO_PI * (double)q / (double)A->n_fft;
        double c = cos(ang), sn = -sin(ang);
        double* e = A->extra + 2 * (i * A->n_f + n);
#pragma omp atomic
        e[0] += vr * c - vi * sn;
#pragma omp atomic
        e[1] += vr * sn + vi * c;
    }
}

/* adjoint of bpa_rc_point: value y at point p over the members perm[b..e).  In the
 * position-gradient mode (A->grad set) each member instead receives
 * Re[conj(y) e^{j 2 k_c R} (j 2 k_c lerp + (P[m0+1] - P[m0]) / dR)] (p'_i - p) / R,
 * the derivative of the BPA-RC term with respect to p'_i paired with y. */
static void bpa_rc_point_adj(adj_prof* A, const double* traj, const i64* perm, i64 b, i64 e, const double p[3],
                             const double y[2]) {
    for (i64 jj = b; jj < e; ++jj) {
        i64 i = perm ? perm[jj] : jj;
        double dx = p[0] - traj[3 * i], dy = p[1] - traj[3 * i + 1], dz = p[2] - traj[3 * i + 2];
        double R = sqrt(dx * dx + dy * dy + dz * dz);
        double mu = R / A->dR;
        double fl = floor(mu);
        double t = mu - fl;
        i64 m0 = (i64)fl;
        double ph = 2.0 * A->kc * R;
        if (A->grad) {
            double a0[2], a1[2];
            prof_get(A->P, i, m0, a0);
            prof_get(A->P, i, m0 + 1, a1);
            double lr = a0[0] + t * (a1[0] - a0[0]), li = a0[1] + t * (a1[1] - a0[1]);
            double Dr = -2.0 * A->kc * li + (a1[0] - a0[0]) / A->dR, Di = 2.0 * A->kc * lr + (a1[1] - a0[1]) / A->dR;
            double c = cos(ph), sn = sin(ph);
            double Er = c * Dr - sn * Di, Ei = c * Di + sn * Dr;
            double coef = (y[0] * Er + y[1] * Ei) / R; /* Re(conj(y) E) / R; p'_i - p = -(dx, dy, dz) */
            double* gi = A->grad + 3 * i;
#pragma omp atomic
            gi[0] -= coef * dx;
#pragma omp atomic
            gi[1] -= coef * dy;
#pragma omp atomic
            gi[2] -= coef * dz;
            continue;
        }
        double cr = cos(ph), ci = -sin(ph);
        double vr = y[0] * cr - y[1] * ci, vi = y[0] * ci + y[1] * cr; /* e^{-j ph} y */
        adj_add_bin(A, i, m0, (1.0 - t) * vr, (1.0 - t) * vi);
        adj_add_bin(A, i, m0 + 1, t * vr, t * vi);
    }
}

typedef struct {
    uint8_t* need;
    uint8_t* feas;  /* needed and feasible (preimage found) */
    double* pre;    /* [N][4]: preimage x, y, z and Phi of the node there */
    double* adj;    /* [N][2]: adjoint values of the samples */
} adj_node;

/* adjoint of child_contrib: value y of f_c at point p */
static void child_contrib_adj(const hho_plan* pl, adj_prof* A, const hho_node* c, adj_node* cd, const double p[3],
                              const double y[2]) {
    footprint F;
    make_footprint(pl, c, p, &F);
    int T = pl->taps, ok = F.inside;
    for (int a = 0; ok && a < T; ++a)
        for (int b = 0; ok && b < T; ++b)
            for (int q = 0; ok && q < T; ++q)
                if (!cd->feas[lat_index(c, F.base[0] + a, F.base[1] + b, F.base[2] + q)]) ok = 0;
    if (!ok) {
        bpa_rc_point_adj(A, pl->traj, pl->perm, c->begin, c->end, p, y);
        return;
    }
    double cr = cos(F.phi), ci = -sin(F.phi);
    double vr = y[0] * cr - y[1] * ci, vi = y[0] * ci + y[1] * cr; /* e^{-j phi_c} y */
    for (int a = 0; a < T; ++a)
        for (int b = 0; b < T; ++b) {
            double wab = F.w[0][a] * F.w[1][b];
            for (int q = 0; q < T; ++q) {
                double ww = wab * F.w[2][q];
                double* o = cd->adj + 2 * lat_index(c, F.base[0] + a, F.base[1] + b, F.base[2] + q);
#pragma omp atomic
                o[0] += ww * vr;
#pragma omp atomic
                o[1] += ww * vi;
            }
        }
}

/* The adjoint's traversal: final level, merges top down, leaves; every BPA-RC
 * term is handed to bpa_rc_point_adj with its value y. */
static void hhffbpa_adjoint_walk(const hho_plan* pl, adj_prof* A, const double* x_ri, const double* pts, i64 n_pts) {
    int nl = pl->n_levels;
    const hho_node* root = &pl->nodes[pl->level_start[nl - 1]];
    if (nl == 1) {
#pragma omp parallel for schedule(dynamic, 16)
        for (i64 q = 0; q < n_pts; ++q)
            bpa_rc_point_adj(A, pl->traj, pl->perm, 0, pl->n_pos, pts + 3 * q, x_ri + 2 * q);
        return;
    }
    {
        adj_node* D = (adj_node*)calloc((size_t)pl->n_nodes, sizeof(adj_node));
        for (i64 k = 0; k < pl->level_start[nl - 1]; ++k) {
            const hho_node* nd = &pl->nodes[k];
            i64 NN = nd->N[0] * nd->N[1] * nd->N[2];
            D[k].need = (uint8_t*)calloc((size_t)NN, 1);
            D[k].feas = (uint8_t*)calloc((size_t)NN, 1);
            D[k].pre = (double*)calloc((size_t)4 * NN, sizeof(double));
            D[k].adj = (double*)calloc((size_t)2 * NN, sizeof(double));
        }
        /* the forward's demand marking, with each needed sample's preimage kept */
        for (i64 c = 0; c < root->nchild; ++c) {
            const hho_node* cn = &pl->nodes[root->child0 + c];
            node_data nd_view = {D[root->child0 + c].need, NULL};
#pragma omp parallel for schedule(dynamic, 64)
            for (i64 q = 0; q < n_pts; ++q) {
                footprint F;
                make_footprint(pl, cn, pts + 3 * q, &F);
                mark_footprint(pl, cn, &nd_view, &F);
            }
        }
        for (int l = nl - 2; l >= 0; --l) {
            for (i64 k = pl->level_start[l]; k < pl->level_start[l + 1]; ++k) {
                const hho_node* nd = &pl->nodes[k];
                i64 NN = nd->N[0] * nd->N[1] * nd->N[2];
#pragma omp parallel for schedule(dynamic, 64)
                for (i64 li = 0; li < NN; ++li) {
                    if (!D[k].need[li]) continue;
                    double tgt[3], p[3];
                    lattice_target(pl, nd, li, tgt);
                    if (!preimage(nd->rect, nd->zbar, pl->kmin, pl->kmax, pl->zh_floor, pl->zh_mid, tgt, p)) continue;
                    double w4[4];
                    uvn_phi(nd->rect, nd->zbar, pl->kmin, pl->kmax, p, w4);
                    D[k].feas[li] = 1;
                    double* pr = D[k].pre + 4 * li;
                    pr[0] = p[0];
                    pr[1] = p[1];
                    pr[2] = p[2];
                    pr[3] = w4[3];
                    if (l == 0) continue;
                    for (i64 c = 0; c < nd->nchild; ++c) {
                        footprint F;
                        node_data nd_view = {D[nd->child0 + c].need, NULL};
                        make_footprint(pl, &pl->nodes[nd->child0 + c], p, &F);
                        mark_footprint(pl, &pl->nodes[nd->child0 + c], &nd_view, &F);
                    }
                }
            }
        }
        /* final level */
#pragma omp parallel for schedule(dynamic, 64)
        for (i64 q = 0; q < n_pts; ++q)
            for (i64 c = 0; c < root->nchild; ++c)
                child_contrib_adj(pl, A, &pl->nodes[root->child0 + c], &D[root->child0 + c], pts + 3 * q,
                                  x_ri + 2 * q);
        /* merges, top down, then the leaves */
        for (int l = nl - 2; l >= 0; --l) {
            for (i64 k = pl->level_start[l]; k < pl->level_start[l + 1]; ++k) {
                const hho_node* nd = &pl->nodes[k];
                i64 NN = nd->N[0] * nd->N[1] * nd->N[2];
#pragma omp parallel for schedule(dynamic, 64)
                for (i64 li = 0; li < NN; ++li) {
                    if (!D[k].feas[li]) continue;
                    const double* pr = D[k].pre + 4 * li;
                    const double* a = D[k].adj + 2 * li;
                    if (a[0] == 0.0 && a[1] == 0.0) continue;
                    double cr = cos(pr[3]), ci = sin(pr[3]);
                    double y[2] = {a[0] * cr - a[1] * ci, a[0] * ci + a[1] * cr}; /* e^{+j Phi} adj */
                    if (l == 0) {
                        bpa_rc_point_adj(A, pl->traj, pl->perm, nd->begin, nd->end, pr, y);
                    } else {
                        for (i64 c = 0; c < nd->nchild; ++c)
                            child_contrib_adj(pl, A, &pl->nodes[nd->child0 + c], &D[nd->child0 + c], pr, y);
                    }
                }
            }
        }
        for (i64 k = 0; k < pl->n_nodes; ++k) {
            free(D[k].need);
            free(D[k].feas);
            free(D[k].pre);
            free(D[k].adj);
        }
        free(D);
    }
}

int hho_hhffbpa_adjoint(const hho_plan* pl, const double* freqs, int n_f, const double* x_ri, const double* pts,
                        i64 n_pts, double* echo_ri) {
    double lo, hi;
    range_bounds(pl->traj, pl->n_pos, pts, n_pts, &lo, &hi);
    hho_prof P; /* the forward's profile window; only its bin range is used here */
    prof_init(&P, NULL, 0, freqs, n_f, pl->os_r, lo - 0.3, hi + 0.3);
    adj_prof A;
    memset(&A, 0, sizeof(A));
    A.n_pos = pl->n_pos;
    A.m_lo = P.m_lo;
    A.n_bins = P.n_bins;
    A.n_f = n_f;
    A.n_fft = P.n_fft;
    A.dR = P.dR;
    A.kc = P.kc;
    A.win = (double*)calloc((size_t)2 * pl->n_pos * P.n_bins, sizeof(double));
    A.extra = (double*)calloc((size_t)2 * pl->n_pos * n_f, sizeof(double));
    prof_free(&P);
    hhffbpa_adjoint_walk(pl, &A, x_ri, pts, n_pts);
    /* range compression: the window's bins transformed, plus the bins outside it */
    double* tab = twiddles(A.n_fft);
    i64 period = 2 * (i64)A.n_fft;
#pragma omp parallel for schedule(static)
    for (i64 i = 0; i < pl->n_pos; ++i)
        for (int n = 0; n < n_f; ++n) {
            double acc[2] = {A.extra[2 * (i * n_f + n)], A.extra[2 * (i * n_f + n) + 1]};
            for (int j = 0; j < A.n_bins; ++j) {
                i64 m = A.m_lo + j;
                i64 mm = ((m % A.n_fft) + A.n_fft) % A.n_fft;
                i64 q = ((i64)(2 * n - n_f + 1) * mm) % period;
                if (q < 0) q += period;
                const double* b = A.win + 2 * (i * A.n_bins + j);
                cmac(acc, b[0], b[1], tab[2 * q], -tab[2 * q + 1]);
            }
            echo_ri[2 * (i * n_f + n)] = acc[0];
            echo_ri[2 * (i * n_f + n) + 1] = acc[1];
        }
    free(tab);
    free(A.win);
    free(A.extra);
    return 0;
}

/* Gradient with respect to the positions of L = Re sum_q conj(x_q) f(p_q), f = HHFFBPA at
 * the points, with the plan (tree, lattices, preimages) held fixed: only the BPA-RC terms of
 * the leaves and of the exact fallbacks depend on the positions.  The adjoint traversal
 * carries each such term's value y; the term's derivative is taken as in the BPA-RC
 * gradient.  grad: [n_pos][3], overwritten. */
int hho_hhffbpa_traj_grad(const hho_plan* pl, const double* freqs, int n_f, const double* echo_ri,
                          const double* x_ri, const double* pts, i64 n_pts, double* grad) {
    double lo, hi;
    range_bounds(pl->traj, pl->n_pos, pts, n_pts, &lo, &hi);
    hho_prof P;
    prof_init(&P, echo_ri, pl->n_pos, freqs, n_f, pl->os_r, lo - 0.3, hi + 0.3);
    adj_prof A;
    memset(&A, 0, sizeof(A));
    A.n_pos = pl->n_pos;
    A.m_lo = P.m_lo;
    A.n_bins = P.n_bins;
    A.n_f = n_f;
    A.n_fft = P.n_fft;
    A.dR = P.dR;
    A.kc = P.kc;
    A.P = &P;
    A.grad = grad;
    memset(grad, 0, sizeof(double) * 3 * (size_t)pl->n_pos);
    hhffbpa_adjoint_walk(pl, &A, x_ri, pts, n_pts);
    prof_free(&P);
    return 0;
}

int hho_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
