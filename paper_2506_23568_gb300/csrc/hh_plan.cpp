// Host planning for HHFFBPA: subarray tree, per-subarray (u, v, n) sampling
// grids, range gate, launch tiles and interpolation weights (Sec. III, Sec. IV-A).
// FP64 throughout; nothing here touches the GPU.
#include <algorithm>
#include <array>
#include <atomic>
#include <condition_variable>
#include <cmath>
#include <cstring>
#include <functional>
#include <mutex>
#include <numeric>
#include <thread>

#include "hh_internal.h"

namespace hh {

namespace {

// Geometry of one subarray for the spectral design of Sec. III.  The design
// plane z' = 0 of the key points is the subarray's mean member height zbar.
struct Sub {
    double a, b, e, g, zbar;
    double kmin, kmax;

    double dist(double x, double y, double zh, double X, double Y) const {
        return std::sqrt((x - X) * (x - X) + (y - Y) * (y - Y) + zh * zh);
    }
    // (u, v, n) of Eq. eq_uvw_xyz and Phi of Eq. eq_sdc_phi at absolute point (x, y, z).
    void uvn(double x, double y, double z, double out[4]) const {
        double zh = z - zbar;
        double xn = std::min(std::max(x, a), b), yn = std::min(std::max(y, e), g);
        double r = dist(x, y, zh, a, e) + dist(x, y, zh, a, g) + dist(x, y, zh, b, e) + dist(x, y, zh, b, g);
        double C2 = 4 * (b - a) * (b - a) + 4 * (g - e) * (g - e);
        double S = std::sqrt(r * r - C2);
        out[0] = kmax / kPi * (dist(x, y, zh, a, yn) - dist(x, y, zh, b, yn));
        out[1] = kmax / kPi * (dist(x, y, zh, xn, e) - dist(x, y, zh, xn, g));
        out[2] = (kmax * S - kmin * r) / (4 * kPi);
        out[3] = 0.25 * (kmax * S + kmin * r);
    }
    // k_0(p', p, k) = 2k (p - p') / |p - p'| (Eq. eq_kfun_posp), p' = (X, Y, Z).
    static void kvec(double X, double Y, double Z, const double p[3], double k, double o[3]) {
        double d[3] = {p[0] - X, p[1] - Y, p[2] - Z};
        double n = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        for (int i = 0; i < 3; ++i) o[i] = 2 * k * d[i] / n;
    }
    // Spectrum centre k_c = (k5 + k7)/2 and the Jacobian rows of (u, v, n):
    // -v1/2pi, -v2/2pi, v3/2pi with v1 = k2-k1, v2 = k4-k3, v3 = k7-k5 (Eq. eq3_lltmatrix).
    void centre_and_jacobian(const double p[3], double kcv[3], double J[3][3]) const {
        double xn = std::min(std::max(p[0], a), b), yn = std::min(std::max(p[1], e), g);
        double k1[3], k2[3], k3[3], k4[3], k5[3] = {0, 0, 0}, t[3];
        kvec(a, yn, zbar, p, kmax, k1);
        kvec(b, yn, zbar, p, kmax, k2);
        kvec(xn, e, zbar, p, kmax, k3);
        kvec(xn, g, zbar, p, kmax, k4);
        const double cx[4] = {a, a, b, b}, cy[4] = {e, g, e, g};
        double r = 0;
        for (int c = 0; c < 4; ++c) {
            kvec(cx[c], cy[c], zbar, p, kmin, t);
            for (int i = 0; i < 3; ++i) k5[i] += 0.25 * t[i];
            r += dist(p[0], p[1], p[2] - zbar, cx[c], cy[c]);
        }
        double C2 = 4 * (b - a) * (b - a) + 4 * (g - e) * (g - e);
        double beta = kmax * r / (kmin * std::sqrt(r * r - C2));  // boresight-matched integrating factor
        for (int i = 0; i < 3; ++i) {
            double k7 = beta * k5[i];
            kcv[i] = 0.5 * (k5[i] + k7);
            J[0][i] = -(k2[i] - k1[i]) / (2 * kPi);
            J[1][i] = -(k4[i] - k3[i]) / (2 * kPi);
            J[2][i] = (k7 - k5[i]) / (2 * kPi);
        }
    }
};

// LU factorisation (partial pivoting) of A^T for a 3x3 A, then solves A^T x = rhs.
struct LU3 {
    double M[3][3];
    int piv[3];
    bool ok;
    explicit LU3(const double A[3][3]) : ok(true) {
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) M[i][j] = A[j][i];
        for (int i = 0; i < 3; ++i) piv[i] = i;
        for (int c = 0; c < 3; ++c) {
            int pr = c;
            for (int r = c + 1; r < 3; ++r)
                if (std::fabs(M[r][c]) > std::fabs(M[pr][c])) pr = r;
            if (!(std::fabs(M[pr][c]) > 0)) {
                ok = false;
                return;
            }
            if (pr != c) {
                for (int j = 0; j < 3; ++j) std::swap(M[c][j], M[pr][j]);
                std::swap(piv[c], piv[pr]);
            }
            for (int r = c + 1; r < 3; ++r) {
                M[r][c] /= M[c][c];
                for (int j = c + 1; j < 3; ++j) M[r][j] -= M[r][c] * M[c][j];
            }
        }
    }
    void solve(const double rhs[3], double x[3]) const {
        double y[3];
        for (int i = 0; i < 3; ++i) {
            double s = rhs[piv[i]];
            for (int j = 0; j < i; ++j) s -= M[i][j] * y[j];
            y[i] = s;
        }
        for (int i = 2; i >= 0; --i) {
            double s = y[i];
            for (int j = i + 1; j < 3; ++j) s -= M[i][j] * x[j];
            x[i] = s / M[i][i];
        }
    }
};

struct GridBox {
    double lo[3], hi[3];
};

GridBox grid_box(const hh_grid& g) {
    GridBox B;
    B.lo[0] = g.x0; B.hi[0] = g.x0 + g.dx * (g.nx - 1);
    B.lo[1] = g.y0; B.hi[1] = g.y0 + g.dy * (g.ny - 1);
    B.lo[2] = g.z0; B.hi[2] = g.z0 + g.dz * (g.nz - 1);
    return B;
}

double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Exact extremes of u, v, n over the box D: u rises with x and is monotone in
// (y - y'_0)^2 + zh^2 on an x-face, so the candidates on the x faces are
// y in {y_lo, y_hi, clamp(e), clamp(g)} x z in {z_lo, z_hi}; v likewise on the
// y faces; n rises with zh and with the corner-distance sum r, which is least at
// the clamped subarray centre and greatest at a corner of the top face.
void uvn_extremes(const Sub& s, const GridBox& B, double mn[3], double mx[3]) {
    double w[4];
    for (int i = 0; i < 3; ++i) {
        mn[i] = HUGE_VAL;
        mx[i] = -HUGE_VAL;
    }
    const double yc[4] = {B.lo[1], B.hi[1], clampd(s.e, B.lo[1], B.hi[1]), clampd(s.g, B.lo[1], B.hi[1])};
    const double xc[4] = {B.lo[0], B.hi[0], clampd(s.a, B.lo[0], B.hi[0]), clampd(s.b, B.lo[0], B.hi[0])};
    for (double z : {B.lo[2], B.hi[2]}) {
        for (int i = 0; i < 4; ++i) {
            s.uvn(B.lo[0], yc[i], z, w); mn[0] = std::min(mn[0], w[0]);
            s.uvn(B.hi[0], yc[i], z, w); mx[0] = std::max(mx[0], w[0]);
            s.uvn(xc[i], B.lo[1], z, w); mn[1] = std::min(mn[1], w[1]);
            s.uvn(xc[i], B.hi[1], z, w); mx[1] = std::max(mx[1], w[1]);
        }
    }
    s.uvn(clampd(0.5 * (s.a + s.b), B.lo[0], B.hi[0]), clampd(0.5 * (s.e + s.g), B.lo[1], B.hi[1]), B.lo[2], w);
    mn[2] = w[2];
    for (double x : {B.lo[0], B.hi[0]})
        for (double y : {B.lo[1], B.hi[1]}) {
            s.uvn(x, y, B.hi[2], w);
            mx[2] = std::max(mx[2], w[2]);
        }
}

// Measured extent of the compressed local spectrum, per (u, v, n) axis, in units
// of the unit box of Eq. eq_llt_spcm_trans.  Probe points: the corners, face
// centres and centre of D.  Spectral components: K = 2k (p - p')/|p - p'|
// (Eq. eq_kxyz_posp) for p' on the subarray border (four points per edge
// starting at each corner, counter-clockwise from (a, e)), at the lowest and
// highest member heights, for k in {k_min, k_max}.  kappa solves J^T kappa = K - k_c.
// Result rounded up to a multiple of 1/64 and at least 1.
void spectral_extent(const Sub& s, double zlo, double zhi, const GridBox& B, double rho[3]) {
    double px[16], py[16];
    for (int q = 0; q < 4; ++q) {
        double f = q / 4.0;
        px[q] = s.a + f * (s.b - s.a); py[q] = s.e;
        px[4 + q] = s.b; py[4 + q] = s.e + f * (s.g - s.e);
        px[8 + q] = s.b - f * (s.b - s.a); py[8 + q] = s.g;
        px[12 + q] = s.a; py[12 + q] = s.g - f * (s.g - s.e);
    }
    rho[0] = rho[1] = rho[2] = 1.0;
    for (int ix = 0; ix < 3; ++ix)
        for (int iy = 0; iy < 3; ++iy)
            for (int iz = 0; iz < 3; ++iz) {
                int mids = (ix == 1) + (iy == 1) + (iz == 1);
                if (mids == 1) continue;  // edge midpoints are not probed
                double p[3] = {ix == 0 ? B.lo[0] : (ix == 2 ? B.hi[0] : 0.5 * (B.lo[0] + B.hi[0])),
                               iy == 0 ? B.lo[1] : (iy == 2 ? B.hi[1] : 0.5 * (B.lo[1] + B.hi[1])),
                               iz == 0 ? B.lo[2] : (iz == 2 ? B.hi[2] : 0.5 * (B.lo[2] + B.hi[2]))};
                double kcv[3], J[3][3];
                s.centre_and_jacobian(p, kcv, J);
                const LU3 lu(J);
                if (!lu.ok) continue;
                for (int q = 0; q < 16; ++q)
                    for (double Z : {zlo, zhi})
                        for (double k : {s.kmin, s.kmax}) {
                            double K[3], rhs[3], kap[3];
                            Sub::kvec(px[q], py[q], Z, p, k, K);
                            for (int i = 0; i < 3; ++i) rhs[i] = K[i] - kcv[i];
                            lu.solve(rhs, kap);
                            for (int i = 0; i < 3; ++i) rho[i] = std::max(rho[i], std::fabs(kap[i]) / kPi);
                        }
            }
    for (int i = 0; i < 3; ++i) rho[i] = std::ceil(rho[i] * 64.0) / 64.0;
}

}  // namespace

void range_constants(const double* freqs, int n_f, int range_os, double* kmin, double* kmax, double* kc,
                     double* dk, int* n_fft, double* dR) {
    *kmin = 2 * kPi * freqs[0] / kC;
    *kmax = 2 * kPi * freqs[n_f - 1] / kC;
    *kc = 0.5 * (*kmin + *kmax);
    *dk = (*kmax - *kmin) / (n_f - 1);
    int64_t want = (int64_t)range_os * n_f;
    int n = 1;
    while (n < want) n <<= 1;
    *n_fft = n;
    *dR = kPi / ((double)n * *dk);
}

int validate_inputs(const double* traj, int64_t n_pos, const double* freqs, int32_t n_f, const hh_grid* grid,
                    const hh_config* cfg, bool need_plan) {
    if (!traj || !freqs || !grid || !cfg) return HH_ERR_ARG;
    if (n_pos < 1 || n_pos > (int64_t)INT32_MAX || n_f < 2) return HH_ERR_ARG;
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return HH_ERR_ARG;
    if (!(grid->dx > 0) || !(grid->dy > 0) || !(grid->dz > 0)) return HH_ERR_ARG;
    if ((int64_t)grid->nx * grid->ny * grid->nz > ((int64_t)1 << 34)) return HH_ERR_ARG;
    if (cfg->range_os < 1 || (int64_t)cfg->range_os * n_f > (1 << 24)) return HH_ERR_ARG;
    for (int64_t i = 0; i < 3 * n_pos; ++i)
        if (!std::isfinite(traj[i])) return HH_ERR_ARG;
    if (!(freqs[0] > 0)) return HH_ERR_FREQ_NONUNIFORM;
    double step = (freqs[n_f - 1] - freqs[0]) / (n_f - 1);
    if (!(step > 0)) return HH_ERR_FREQ_NONUNIFORM;
    for (int n = 0; n < n_f; ++n) {
        double want = freqs[0] + step * n;
        if (!std::isfinite(freqs[n]) || std::fabs(freqs[n] - want) > 1e-9 * std::fabs(want))
            return HH_ERR_FREQ_NONUNIFORM;
    }
    if (need_plan) {
        if (cfg->leaf_size < 1) return HH_ERR_ARG;
        if (cfg->merge_factor != 2 && cfg->merge_factor != 4) return HH_ERR_ARG;
        if (!(cfg->eta >= 1.0f) || cfg->eta > 16.0f) return HH_ERR_ARG;
        if (cfg->taps != 4 && cfg->taps != 6) return HH_ERR_ARG;
        double ztop = -HUGE_VAL;
        for (int64_t i = 0; i < n_pos; ++i) ztop = std::max(ztop, traj[3 * i + 2]);
        if (!(grid->z0 > ztop)) return HH_ERR_ARG;  // D must lie in front of every position
    }
    return HH_OK;
}

std::vector<float> twiddle_table(int n_fft) {
    // W[q] = exp(+j pi q / n_fft), q in [0, 2 n_fft); computed once per size and kept
    // (every plan of a scan series uses the same transform length)
    static std::mutex mu;
    static std::vector<std::pair<int, std::vector<float>>> cache;
    {
        std::lock_guard<std::mutex> lk(mu);
        for (const auto& e : cache)
            if (e.first == n_fft) return e.second;
    }
    std::vector<float> t(4 * (size_t)n_fft);
    for (int q = 0; q < 2 * n_fft; ++q) {
        double ang = kPi * (double)q / (double)n_fft;
        t[2 * q] = (float)std::cos(ang);
        t[2 * q + 1] = (float)std::sin(ang);
    }
    std::lock_guard<std::mutex> lk(mu);
    if (cache.size() < 16) cache.emplace_back(n_fft, t);
    return t;
}

// Solves the n x n system A x = b in place (Gauss-Jordan, partial pivoting);
// a is row-major n x (n + 1) with b in the last column, x left there.
static void solve_augmented(std::vector<double>& a, int n) {
    const int w = n + 1;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(a[r * w + c]) > std::fabs(a[piv * w + c])) piv = r;
        if (piv != c)
            for (int j = 0; j <= n; ++j) std::swap(a[c * w + j], a[piv * w + j]);
        const double d = a[c * w + c];
        for (int j = 0; j <= n; ++j) a[c * w + j] /= d;
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const double f = a[r * w + c];
            for (int j = 0; j <= n; ++j) a[r * w + j] -= f * a[c * w + j];
        }
    }
}

// Least-squares fractional-delay weights for a flat spectrum on |f| <= 1/(2 eta)
// cycles/sample (the unit box sampled at density eta): taps at offsets
// -(T/2-1) .. T/2, h(tau) = G^-1 r(tau), G_ij = sinc((o_i - o_j)/eta),
// r_i = sinc((o_i - tau)/eta).
static void ls_weights(int taps, double eta, double tau, double* h) {
    auto sinc = [](double x) { return x == 0.0 ? 1.0 : std::sin(kPi * x) / (kPi * x); };
    const int o0 = -(taps / 2 - 1);
    std::vector<double> a((size_t)taps * (taps + 1));
    for (int i = 0; i < taps; ++i) {
        for (int j = 0; j < taps; ++j) a[i * (taps + 1) + j] = sinc((double)(i - j) / eta);
        a[i * (taps + 1) + taps] = sinc(((double)(o0 + i) - tau) / eta);
    }
    solve_augmented(a, taps);
    for (int i = 0; i < taps; ++i) h[i] = a[i * (taps + 1) + taps];
}

// The weights as degree-8 polynomials of x = 2 tau - 1: interpolation of
// h_q(tau) at the 9 Chebyshev nodes of [-1, 1] (within about 1e-7 of the exact
// weights everywhere, the FP32 rounding level), split into even and odd parts.
WPoly weight_poly(int taps, double eta) {
    constexpr int kDeg = 8, kN = kDeg + 1;
    WPoly wp{};
    std::vector<double> h((size_t)kN * taps);
    double xs[kN];
    for (int k = 0; k < kN; ++k) {
        xs[k] = std::cos((2 * k + 1) * kPi / (2 * kN));
        ls_weights(taps, eta, 0.5 * (xs[k] + 1.0), &h[(size_t)k * taps]);
    }
    for (int q = 0; q < taps / 2 && q < kPolyPairs; ++q) {
        std::vector<double> a((size_t)kN * (kN + 1));  // Vandermonde system for the monomial coefficients
        for (int k = 0; k < kN; ++k) {
            double xp = 1.0;
            for (int j = 0; j < kN; ++j, xp *= xs[k]) a[k * (kN + 1) + j] = xp;
            a[k * (kN + 1) + kN] = h[(size_t)k * taps + q];
        }
        solve_augmented(a, kN);
        for (int j = 0; j < kN; ++j) {
            const float c = (float)a[j * (kN + 1) + kN];
            if (j % 2 == 0) wp.e[q][j / 2] = c;
            else wp.o[q][j / 2] = c;
        }
    }
    return wp;
}

namespace {

// Host workers kept for the life of the process, so that the planner's parallel loops
// (a few per plan, each well under a millisecond of work) do not pay for creating
// threads.  One loop runs at a time; a call that finds the workers busy (another host
// thread, or a loop inside a loop) runs on threads of its own instead.
class WorkerPool {
  public:
    explicit WorkerPool(int n) {
        for (int i = 0; i < n; ++i) workers_.emplace_back([this]() { work(); });
    }
    ~WorkerPool() {
        {
            std::lock_guard<std::mutex> lk(mu_);
            stop_ = true;
        }
        cv_.notify_all();
        for (auto& w : workers_) w.join();
    }
    int size() const { return (int)workers_.size(); }
    // Runs f(i) for i in [0, n) on the calling thread and up to `helpers` workers; false
    // (nothing run) when the pool is in use.
    bool run(int64_t n, int helpers, const std::function<void(int64_t)>& f) {
        std::unique_lock<std::mutex> busy(call_mu_, std::try_to_lock);
        if (!busy.owns_lock()) return false;
        {
            std::lock_guard<std::mutex> lk(mu_);
            job_ = &f;
            n_ = n;
            next_.store(0);
            want_ = helpers;
            pending_ = 0;
            ++gen_;
            gen_pub_.store(gen_, std::memory_order_release);
        }
        cv_.notify_all();
        drain(f, n);
        std::unique_lock<std::mutex> lk(mu_);
        want_ = 0;  // late workers of this generation take nothing
        done_cv_.wait(lk, [this]() { return pending_ == 0; });
        job_ = nullptr;
        return true;
    }

  private:
    void drain(const std::function<void(int64_t)>& f, int64_t n) {
        for (int64_t i = next_.fetch_add(1); i < n; i = next_.fetch_add(1)) f(i);
    }
    // A worker polls for the next job for a short while before it sleeps: the plan's
    // parallel loops follow one another within microseconds, and a wake-up through the
    // condition variable costs tens of microseconds per loop.
    void work() {
        uint64_t seen = 0;
        for (;;) {
            for (int i = 0; i < kPollIters && gen_pub_.load(std::memory_order_acquire) == seen; ++i) {
            }
            std::unique_lock<std::mutex> lk(mu_);
            cv_.wait(lk, [&]() { return stop_ || gen_ != seen; });
            if (stop_) return;
            seen = gen_;
            if (want_ <= 0 || job_ == nullptr) continue;
            --want_;
            ++pending_;
            const std::function<void(int64_t)>* f = job_;
            const int64_t n = n_;
            lk.unlock();
            drain(*f, n);
            lk.lock();
            if (--pending_ == 0) done_cv_.notify_all();
        }
    }
    static constexpr int kPollIters = 1 << 18;
    std::vector<std::thread> workers_;
    std::atomic<uint64_t> gen_pub_{0};
    std::mutex mu_, call_mu_;
    std::condition_variable cv_, done_cv_;
    const std::function<void(int64_t)>* job_ = nullptr;
    int64_t n_ = 0;
    std::atomic<int64_t> next_{0};
    int want_ = 0, pending_ = 0;
    uint64_t gen_ = 0;
    bool stop_ = false;
};

WorkerPool& worker_pool() {
    static WorkerPool pool(std::max(0, std::min(31, (int)std::thread::hardware_concurrency() - 1)));
    return pool;
}

}  // namespace

void parallel_for(int64_t n, int threads, const std::function<void(int64_t)>& f) {
    const int64_t hw = std::max<int64_t>(1, (int64_t)std::thread::hardware_concurrency());
    const int64_t nt = std::max<int64_t>(1, std::min<int64_t>({hw, (int64_t)threads, n}));
    if (nt == 1) {
        for (int64_t i = 0; i < n; ++i) f(i);
        return;
    }
    WorkerPool& wp = worker_pool();
    if (wp.size() > 0 && wp.run(n, (int)std::min<int64_t>(nt - 1, wp.size()), f)) return;
    std::vector<std::thread> pool;
    for (int64_t t = 1; t < nt; ++t)
        pool.emplace_back([&f, n, nt, t]() {
            for (int64_t i = t; i < n; i += nt) f(i);
        });
    for (int64_t i = 0; i < n; i += nt) f(i);
    for (auto& th : pool) th.join();
}

// Moves the `need` smallest members of idx[0, n) in (coordinate along `axis`, index)
// order to the front and the rest behind them (order within each part as found).  The
// coordinates are binned by a monotone map onto equal-width buckets between their minimum
// and maximum, so that every bucket below the one holding the boundary lies wholly in
// front and every bucket above it wholly behind; only that bucket is ordered exactly.
// Linear time; the partition equals that of a full sort.
void select_lower(const double* T, int axis, int64_t* idx, int64_t n, int64_t need) {
    auto less = [T, axis](int64_t u, int64_t v) {
        const double cu = T[3 * u + axis], cv = T[3 * v + axis];
        return cu < cv || (cu == cv && u < v);
    };
    if (need <= 0 || need >= n) return;
    constexpr int kBins = 4096;
    if (n < 4 * kBins / 16) {
        std::nth_element(idx, idx + need, idx + n, less);
        return;
    }
    double lo4[4] = {HUGE_VAL, HUGE_VAL, HUGE_VAL, HUGE_VAL}, hi4[4] = {-HUGE_VAL, -HUGE_VAL, -HUGE_VAL, -HUGE_VAL};
    for (int64_t q = 0; q < n; ++q) {  // four independent chains
        const double x = T[3 * idx[q] + axis];
        lo4[q & 3] = x < lo4[q & 3] ? x : lo4[q & 3];
        hi4[q & 3] = x > hi4[q & 3] ? x : hi4[q & 3];
    }
    const double lo = std::min(std::min(lo4[0], lo4[1]), std::min(lo4[2], lo4[3]));
    const double hi = std::max(std::max(hi4[0], hi4[1]), std::max(hi4[2], hi4[3]));
    const double scale = (double)kBins / (hi - lo);
    if (!(hi > lo) || !std::isfinite(scale)) {
        std::nth_element(idx, idx + need, idx + n, less);
        return;
    }
    thread_local std::vector<uint16_t> bin;
    thread_local std::vector<int64_t> out, cand;
    bin.resize(n);
    out.resize(n + 1);  // the branch-free partition below writes one slot past each part
    int64_t count[kBins] = {0};
    for (int64_t q = 0; q < n; ++q) {
        const int b = std::min(kBins - 1, (int)((T[3 * idx[q] + axis] - lo) * scale));
        bin[q] = (uint16_t)b;
        ++count[b];
    }
    int kb = 0;
    int64_t below = 0;
    while (below + count[kb] < need) below += count[kb++];
    cand.resize(count[kb] + 1);
    int64_t L = 0, R = need, C = 0;
    int64_t* o = out.data();
    int64_t* c = cand.data();
    for (int64_t q = 0; q < n; ++q) {  // every member is written to all three parts; only its own advances
        const int64_t id = idx[q];
        const int b = bin[q];
        o[L] = id;
        o[R] = id;
        c[C] = id;
        L += b < kb;
        R += b > kb;
        C += b == kb;
    }
    const int64_t take = need - below;
    std::nth_element(c, c + take, c + C, less);
    for (int64_t i = 0; i < C; ++i) o[i < take ? L++ : R++] = c[i];
    std::copy(out.begin(), out.begin() + n, idx);
}

int build_host_plan(hh_plan* p) {
    const hh_config& cfg = p->cfg;
    const int64_t n = p->n_pos;
    const double* T = p->traj.data();
    range_constants(p->freqs.data(), p->n_f, cfg.range_os, &p->kmin, &p->kmax, &p->kc, &p->dk, &p->n_fft, &p->dR);
    double zsum = 0, ztop = -HUGE_VAL;
    for (int64_t i = 0; i < n; ++i) {
        zsum += T[3 * i + 2];
        ztop = std::max(ztop, T[3 * i + 2]);
    }
    p->zbar_all = zsum / (double)n;
    p->zh_floor = 0.1 * (p->grid.z0 - ztop);
    const GridBox B = grid_box(p->grid);
    const double min_ext = 0.5 * kC / p->freqs[p->n_f - 1];  // half the shortest wavelength

    // ---- binary k-d tree (Sec. IV-A: 2^(M-1) level-1 subarrays; the split
    // rule for arbitrary tracks is ours): depth d halves each node along x (d
    // even) or y (d odd) in (coordinate, index) order, the lower part taking
    // floor(n/2) members.
    int D = 0;
    while (((int64_t)1 << (D + 1)) * (int64_t)cfg.leaf_size <= n) ++D;
    p->depth_leaves = D;
    p->perm.resize(n);
    std::iota(p->perm.begin(), p->perm.end(), (int64_t)0);
    // node boundaries depend on the sizes alone
    std::vector<std::vector<int64_t>> bounds(D + 1);
    bounds[0] = {0, n};
    for (int d = 0; d < D; ++d) {
        const std::vector<int64_t>& bd = bounds[d];
        std::vector<int64_t>& nb = bounds[d + 1];
        for (size_t j = 0; j + 1 < bd.size(); ++j) {
            nb.push_back(bd[j]);
            nb.push_back(bd[j] + (bd[j + 1] - bd[j]) / 2);
        }
        nb.push_back(n);
    }
    // the selections: node j of depth d splits at its mid point.  The nodes of one depth
    // are independent and run on the host workers; each range sees the same operations
    // whichever thread runs it.
    for (int d = 0; d < D; ++d) {
        const int64_t cnt = (int64_t)1 << d;
        parallel_for(cnt, cnt >= 2 ? 16 : 1, [&](int64_t j) {
            const int64_t b0 = bounds[d][j], b1 = bounds[d][j + 1];
            select_lower(T, d & 1, p->perm.data() + b0, b1 - b0, (b1 - b0) / 2);
        });
    }
    // materialised depths: D, D - s, ..., (> 0), then the root
    const int step = cfg.merge_factor == 4 ? 2 : 1;
    std::vector<int> depths;
    for (int d = D; d > 0; d -= step) depths.push_back(d);
    depths.push_back(0);
    p->n_levels = (int)depths.size();
    if (p->n_levels > kMaxLevels) return HH_ERR_ARG;
    p->level_start.assign(p->n_levels + 1, 0);
    p->nodes.clear();
    for (int l = 0; l < p->n_levels; ++l) {
        p->level_start[l] = (int64_t)p->nodes.size();
        const int d = depths[l];
        const int64_t cnt = (int64_t)1 << d;
        for (int64_t j = 0; j < cnt; ++j) {
            HNode nd;
            nd.level = l;
            nd.depth = d;
            nd.t = p->n_levels - 1 - l;
            nd.begin = bounds[d][j];
            nd.end = bounds[d][j + 1];
            if (l > 0) {
                const int64_t f = (int64_t)1 << (depths[l - 1] - d);
                nd.child0 = p->level_start[l - 1] + j * f;
                nd.nchild = f;
            }
            p->nodes.push_back(nd);
        }
    }
    p->level_start[p->n_levels] = (int64_t)p->nodes.size();
    // member boxes and height sums: the leaves from their members (one leaf per task), every
    // other node as the union of its children's (the same minima and maxima)
    std::vector<std::array<double, 7>> raw(p->nodes.size());  // x min, x max, y min, y max, z min, z max, z sum
    parallel_for(p->level_start[1] - p->level_start[0], n >= 32768 ? 16 : 1, [&](int64_t k) {
        const HNode& nd = p->nodes[k];
        std::array<double, 7> r = {HUGE_VAL, -HUGE_VAL, HUGE_VAL, -HUGE_VAL, HUGE_VAL, -HUGE_VAL, 0.0};
        for (int64_t q = nd.begin; q < nd.end; ++q) {
            const double* pp = T + 3 * p->perm[q];
            r[0] = std::min(r[0], pp[0]); r[1] = std::max(r[1], pp[0]);
            r[2] = std::min(r[2], pp[1]); r[3] = std::max(r[3], pp[1]);
            r[4] = std::min(r[4], pp[2]); r[5] = std::max(r[5], pp[2]);
            r[6] += pp[2];
        }
        raw[k] = r;
    });
    for (int l = 1; l < p->n_levels; ++l)
        for (int64_t k = p->level_start[l]; k < p->level_start[l + 1]; ++k) {
            const HNode& nd = p->nodes[k];
            std::array<double, 7> r = raw[nd.child0];
            for (int64_t c = 1; c < nd.nchild; ++c) {
                const std::array<double, 7>& o = raw[nd.child0 + c];
                for (int i = 0; i < 6; i += 2) {
                    r[i] = std::min(r[i], o[i]);
                    r[i + 1] = std::max(r[i + 1], o[i + 1]);
                }
                r[6] += o[6];
            }
            raw[k] = r;
        }
    for (size_t k = 0; k < p->nodes.size(); ++k) {
        HNode& nd = p->nodes[k];
        const std::array<double, 7>& r = raw[k];
        double a = r[0], b = r[1], e = r[2], g = r[3];
        nd.zmin = r[4];
        nd.zmax = r[5];
        nd.zbar = r[6] / (double)(nd.end - nd.begin);
        if (b - a < min_ext) { double c = 0.5 * (a + b); a = c - 0.5 * min_ext; b = c + 0.5 * min_ext; }
        if (g - e < min_ext) { double c = 0.5 * (e + g); e = c - 0.5 * min_ext; g = c + 0.5 * min_ext; }
        nd.rect[0] = a; nd.rect[1] = b; nd.rect[2] = e; nd.rect[3] = g;
    }

    // ---- sampling grids: a uniform lattice in (u, v, n) per non-root node
    // (Sec. IV-A), covering the image of D plus a margin, with per-axis density
    // eta * rho (rho: measured spectral extent).  The margin is the footprint
    // reach m = taps/2 times the merges above the node for n, and the same
    // capped at 2m for u, v with 4-way merges (their steps halve per level);
    // plus one step.
    const int64_t m = cfg.taps / 2;
    const int64_t n_lattice_nodes = p->level_start[p->n_levels - 1];
    auto lattice_of = [&](int64_t k) {
        HNode& nd = p->nodes[k];
        Sub s{nd.rect[0], nd.rect[1], nd.rect[2], nd.rect[3], nd.zbar, p->kmin, p->kmax};
        double mn[3], mx[3], rho[3];
        uvn_extremes(s, B, mn, mx);
        spectral_extent(s, nd.zmin, nd.zmax, B, rho);
        const int64_t pad_n = m * nd.t + 1;
        const int64_t pad_uv = cfg.merge_factor == 4 ? std::min(m * nd.t, 2 * m) + 1 : pad_n;
        const int64_t pad[3] = {pad_uv, pad_uv, pad_n};
        for (int i = 0; i < 3; ++i) {
            nd.eta[i] = (double)cfg.eta * rho[i];
            nd.lo[i] = mn[i] - (double)pad[i] / nd.eta[i];
            nd.N[i] = (int64_t)std::ceil((mx[i] - mn[i]) * nd.eta[i]) + 1 + 2 * pad[i];
        }
    };
    // nodes are independent: spread them over the host threads (same results in any split)
    parallel_for(n_lattice_nodes, n_lattice_nodes >= 8 ? 32 : 1, lattice_of);
    p->level_samples.assign(p->n_levels, 0);
    p->max_pool = 0;
    for (int l = 0; l + 1 < p->n_levels; ++l) {
        int64_t off = 0;
        for (int64_t k = p->level_start[l]; k < p->level_start[l + 1]; ++k) {
            HNode& nd = p->nodes[k];
            nd.pool_off = off;
            off += nd.N[0] * nd.N[1] * nd.N[2];
        }
        p->level_samples[l] = off;
        p->max_pool = std::max(p->max_pool, off);
    }
    p->level_samples[p->n_levels - 1] = (int64_t)p->grid.nx * p->grid.ny * p->grid.nz;
    p->need_base.assign(p->n_levels, 0);
    p->xyz_base.assign(p->n_levels, 0);
    p->need_total = p->xyz_total = 0;
    for (int l = 0; l + 1 < p->n_levels; ++l) {  // leaves too: the adjoint stores their preimages
        p->xyz_base[l] = p->xyz_total;
        p->xyz_total += p->level_samples[l];
    }

    // ---- range gate: bins covering every range a kernel can look up.  For a
    // lattice of n in [n_lo, n_hi], the corner-distance sum r obeys
    // 4 pi n <= (kmax - kmin) r  and  (kmax - kmin) r^2 - 4 pi n r - kmax C^2 <= 0,
    // each corner distance lies within r/4 -/+ the subarray diagonal and each
    // member within the diagonal plus its height offset of a corner.  D's own
    // ranges (final level and direct BPA) are added.
    double Rlo = HUGE_VAL, Rhi = 0;
    {
        double smin = 0, smax = 0;
        for (int i = 0; i < 3; ++i) {
            double tl = HUGE_VAL, th = -HUGE_VAL;
            for (int64_t q = 0; q < n; ++q) { tl = std::min(tl, T[3 * q + i]); th = std::max(th, T[3 * q + i]); }
            double gap = std::max(0.0, std::max(B.lo[i] - th, tl - B.hi[i]));
            double span = std::max(std::fabs(B.hi[i] - tl), std::fabs(th - B.lo[i]));
            smin += gap * gap;
            smax += span * span;
        }
        Rlo = std::sqrt(smin);
        Rhi = std::sqrt(smax);
    }
    const double dkk = p->kmax - p->kmin;
    for (int l = 0; l + 1 < p->n_levels; ++l)
        for (int64_t k = p->level_start[l]; k < p->level_start[l + 1]; ++k) {
            const HNode& nd = p->nodes[k];
            double C2 = 4 * ((nd.rect[1] - nd.rect[0]) * (nd.rect[1] - nd.rect[0]) +
                             (nd.rect[3] - nd.rect[2]) * (nd.rect[3] - nd.rect[2]));
            double diag = std::sqrt(C2) / 2;
            double nlo = nd.lo[2], nhi = nd.lo[2] + (double)(nd.N[2] - 1) / nd.eta[2];
            double rmin = std::max(std::sqrt(C2), 4 * kPi * nlo / dkk);
            double rmax = (4 * kPi * nhi + std::sqrt(16 * kPi * kPi * nhi * nhi + 4 * dkk * p->kmax * C2)) / (2 * dkk);
            double dz = std::max(std::fabs(nd.zmax - nd.zbar), std::fabs(nd.zmin - nd.zbar));
            Rlo = std::min(Rlo, std::max(0.0, rmin / 4 - 2 * diag - dz));
            Rhi = std::max(Rhi, rmax / 4 + 2 * diag + dz);
        }
    p->gate0 = (int64_t)std::floor(Rlo / p->dR) - 2;
    p->gate_n = (int64_t)std::ceil(Rhi / p->dR) + 3 - p->gate0;
    p->gate_wrap = false;
    if (p->gate_n >= p->n_fft) {
        p->gate0 = 0;
        p->gate_n = p->n_fft;
        p->gate_wrap = true;
    }

    // ---- launch tiles: kTile0 x kTile1 x kTile2 boxes of each node's lattice, and of the grid
    p->level_tiles.assign(p->n_levels, 0);
    p->tile_off.clear();
    p->tile_off_base.assign(p->n_levels, 0);
    for (int l = 0; l + 1 < p->n_levels; ++l) {
        p->tile_off_base[l] = (int64_t)p->tile_off.size();
        int64_t t = 0;
        for (int64_t k = p->level_start[l]; k < p->level_start[l + 1]; ++k) {
            const HNode& nd = p->nodes[k];
            p->tile_off.push_back(t);
            t += ((nd.N[0] + kTile0 - 1) / kTile0) * ((nd.N[1] + kTile1 - 1) / kTile1) *
                 ((nd.N[2] + kTile2 - 1) / kTile2);
        }
        p->tile_off.push_back(t);
        p->level_tiles[l] = t;
    }
    // tile pairs of the merge launches: two launch tiles adjacent along n in one (u, v)
    // column of a node (the last tile of a column alone when the column has an odd count)
    p->level_pairs.assign(p->n_levels, 0);
    p->pair_off.clear();
    p->pair_off_base.assign(p->n_levels, 0);
    for (int l = 0; l + 1 < p->n_levels; ++l) {
        p->pair_off_base[l] = (int64_t)p->pair_off.size();
        int64_t t = 0;
        for (int64_t k = p->level_start[l]; k < p->level_start[l + 1]; ++k) {
            const HNode& nd = p->nodes[k];
            p->pair_off.push_back(t);
            const int64_t nt2 = (nd.N[2] + kTile2 - 1) / kTile2;
            t += ((nd.N[0] + kTile0 - 1) / kTile0) * ((nd.N[1] + kTile1 - 1) / kTile1) * ((nt2 + 1) / 2);
        }
        p->pair_off.push_back(t);
        p->level_pairs[l] = t;
    }
    {
        const hh_grid& g = p->grid;
        p->level_tiles[p->n_levels - 1] = (int64_t)((g.nx + kTile0 - 1) / kTile0) * ((g.ny + kTile1 - 1) / kTile1) *
                                          ((g.nz + kTile2 - 1) / kTile2);
    }
    // need masks: one bit per lattice sample, 256 bits (eight words) per launch tile
    for (int l = 0; l + 1 < p->n_levels; ++l) {
        p->need_base[l] = p->need_total;
        p->need_total += kNeedWords * p->level_tiles[l];
    }
    p->wpoly = weight_poly(cfg.taps, cfg.eta);
    return HH_OK;
}

}  // namespace hh
