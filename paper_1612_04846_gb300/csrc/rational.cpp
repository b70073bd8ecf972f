// Best uniform rational approximation of t^(1-alpha) on [0,1] in R(k,k) (host setup step).
//
// What it computes (Sec. 2.1-2.2): r = P_k/Q_k minimising max_[0,1] |t^(1-alpha) - r(t)|, which
// by Lemma BURA_caracter has real negative interlacing zeros zeta_j and poles d_j and 2k+2
// alternation points 0 = eta_1 < ... < eta_{2k+2} = 1 with t^(1-alpha) - r(eta_i) = (-1)^i E.
// Output: the coefficients of t^{-1} r(t) = sum_{j=0}^k c_j/(t - d_j), d_0 = 0 (eq. (simplified)).
//
// How (differs from Algorithm 1 of Sec. 3.2 by design): the paper solves the linearised
// equioscillation system in a Chebyshev basis, which needs quad precision and stops converging
// near k = 7..11 (Table tabLastS) because the alternation points cluster at t = 0.  Here r is kept
// in factored form r(t) = exp(l) prod_j (t + e^{u_j}) / (t + e^{w_j}); every factor is evaluated
// to full relative precision in double for t >= 0, so no extra precision is needed.
//   * For a fixed reference set the 2k+2 equations t_i^(1-alpha) - r(t_i) - (-1)^i E = 0 are solved
//     for (l, u, w, E) by damped Newton with the exact Jacobian.
//   * The reference is moved to the local extrema of the error between its zeros (Remez exchange;
//     zeros by bisection in log t, maxima by golden-section search in log t).
//   * Start: the k = 1 problem at alpha = 1/2 from a fixed guess, continuation in k at alpha = 1/2
//     (one new zero/pole pair and two reference points extrapolated below the smallest ones),
//     then continuation in alpha with an adaptive step to the requested alpha.
//   * Warm start: the converged states on a fixed grid of alpha (steps of kGridStep) are kept per k,
//     each reached from the alpha = 1/2 anchor exactly as a cold start; a requested alpha continues
//     from the nearest grid state.  The result is a function of (alpha, k) alone, whatever was
//     solved before in the process.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "../../include/bura.h"

namespace {

struct Rat {
    int k = 0;
    std::vector<double> th;  // th[0] = l, th[1..k] = u (zeros), th[k+1..2k] = w (poles)
    std::vector<double> T;   // 2k+2 reference points
    double E = 0;
};

inline double rval(const Rat& R, double t) {
    double v = std::exp(R.th[0]);
    for (int j = 0; j < R.k; ++j) v *= (t + std::exp(R.th[1 + j])) / (t + std::exp(R.th[1 + R.k + j]));
    return v;
}

inline double errval(const Rat& R, double g, double t) { return (t > 0 ? std::pow(t, g) : 0.0) - rval(R, t); }

// Gaussian elimination with partial pivoting; returns false when singular.
bool dense_solve(std::vector<double>& A, std::vector<double>& b, int n) {
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[r * n + c]) > std::fabs(A[p * n + c])) p = r;
        if (!(std::fabs(A[p * n + c]) > 0)) return false;
        if (p != c) {
            for (int j = 0; j < n; ++j) std::swap(A[p * n + j], A[c * n + j]);
            std::swap(b[p], b[c]);
        }
        for (int r = c + 1; r < n; ++r) {
            double f = A[r * n + c] / A[c * n + c];
            if (f == 0) continue;
            for (int j = c; j < n; ++j) A[r * n + j] -= f * A[c * n + j];
            b[r] -= f * b[c];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = b[r];
        for (int j = r + 1; j < n; ++j) s -= A[r * n + j] * b[j];
        b[r] = s / A[r * n + r];
    }
    return true;
}

double residual_norm(const Rat& R, double g, double E, std::vector<double>* F) {
    const int l = 2 * R.k + 2;
    double s = 0;
    for (int i = 0; i < l; ++i) {
        double sg = (i % 2 == 0) ? -1.0 : 1.0;  // (-1)^i with i = 1..l
        double v = errval(R, g, R.T[i]) - sg * E;
        if (F) (*F)[i] = v;
        s += v * v;
    }
    return std::sqrt(s);
}

// Newton on the equioscillation equations for the current reference; false on failure.
bool newton(Rat& R, double g, double& E) {
    const int k = R.k, l = 2 * k + 2;
    std::vector<double> F(l), J(l * l), dx(l);
    double nf = residual_norm(R, g, E, &F);
    for (int it = 0; it < 40; ++it) {
        for (int i = 0; i < l; ++i) {
            const double t = R.T[i];
            const double r = rval(R, t);
            double* Ji = &J[i * l];
            Ji[0] = -r;
            for (int j = 0; j < k; ++j) {
                const double zu = std::exp(R.th[1 + j]), zw = std::exp(R.th[1 + k + j]);
                Ji[1 + j] = -r * zu / (t + zu);
                Ji[1 + k + j] = r * zw / (t + zw);
            }
            Ji[l - 1] = (i % 2 == 0) ? 1.0 : -1.0;  // d/dE of -(-1)^i E
        }
        for (int i = 0; i < l; ++i) dx[i] = -F[i];
        std::vector<double> Jc = J;
        if (!dense_solve(Jc, dx, l)) return false;
        double lam = 1.0;
        Rat trial = R;
        double En = E, nfn = 0;
        bool ok = false;
        while (lam > 1e-4) {
            for (int j = 0; j < l - 1; ++j) trial.th[j] = R.th[j] + lam * dx[j];
            En = E + lam * dx[l - 1];
            nfn = residual_norm(trial, g, En, nullptr);
            if (std::isfinite(nfn) && (nfn < nf || nfn < 1e-17)) { ok = true; break; }
            lam *= 0.5;
        }
        if (!ok) break;
        double step = 0;
        for (int j = 0; j < l; ++j) step = std::max(step, std::fabs(lam * dx[j]));
        R.th = trial.th;
        E = En;
        nf = residual_norm(R, g, E, &F);
        if (step < 1e-14) break;
    }
    return std::isfinite(nf) && nf <= 1e-3 * std::fabs(E);
}

double golden_max(const Rat& R, double g, double a, double b) {
    const double gr = 0.5 * (std::sqrt(5.0) - 1.0);
    double x1 = b - gr * (b - a), x2 = a + gr * (b - a);
    double f1 = std::fabs(errval(R, g, std::exp(x1))), f2 = std::fabs(errval(R, g, std::exp(x2)));
    while (b - a > 1e-13 * std::max(1.0, std::fabs(a))) {
        if (f1 > f2) { b = x2; x2 = x1; f2 = f1; x1 = b - gr * (b - a); f1 = std::fabs(errval(R, g, std::exp(x1))); }
        else { a = x1; x1 = x2; f1 = f2; x2 = a + gr * (b - a); f2 = std::fabs(errval(R, g, std::exp(x2))); }
    }
    return 0.5 * (a + b);
}

// Remez exchange: new reference at the error extrema between consecutive zeros.
bool exchange(Rat& R, double g) {
    const int l = 2 * R.k + 2;
    std::vector<double> es(l);
    for (int i = 0; i < l; ++i) es[i] = errval(R, g, R.T[i]);
    for (int i = 0; i + 1 < l; ++i)
        if ((es[i] > 0) == (es[i + 1] > 0)) return false;
    std::vector<double> bnd(l + 1);
    bnd[0] = 0.0;
    bnd[l] = 1.0;
    for (int i = 0; i + 1 < l; ++i) {
        double a = R.T[i], b = R.T[i + 1], ea = es[i];
        for (int it = 0; it < 200; ++it) {
            double m = a > 0 ? std::sqrt(a * b) : b * 1e-3;
            double em = errval(R, g, m);
            if ((em > 0) == (ea > 0)) { a = m; ea = em; } else b = m;
            if (a > 0 && b / a - 1 < 1e-15) break;
        }
        bnd[i + 1] = 0.5 * (a + b);
    }
    std::vector<double> nT(l);
    nT[0] = 0.0;
    nT[l - 1] = 1.0;
    for (int i = 1; i + 1 < l; ++i) {
        const double la = std::log(bnd[i]), lb = std::log(bnd[i + 1]);
        const int ns = 16;
        int best = 0;
        double bv = -1;
        for (int s = 0; s <= ns; ++s) {
            double v = std::fabs(errval(R, g, std::exp(la + (lb - la) * s / ns)));
            if (v > bv) { bv = v; best = s; }
        }
        double a = la + (lb - la) * std::max(best - 1, 0) / ns;
        double b = la + (lb - la) * std::min(best + 1, ns) / ns;
        nT[i] = std::exp(golden_max(R, g, a, b));
    }
    R.T = nT;
    return true;
}

bool remez(Rat& R, double alpha) {
    const double g = 1.0 - alpha;
    double E = std::fabs(errval(R, g, 0.0));
    const int l = 2 * R.k + 2;
    double spread = 1e300;
    for (int n = 0; n < 40; ++n) {
        if (!newton(R, g, E)) return false;
        if (!exchange(R, g)) return false;
        double mx = 0, mn = 1e300;
        for (int i = 0; i < l; ++i) {
            double v = std::fabs(errval(R, g, R.T[i]));
            mx = std::max(mx, v);
            mn = std::min(mn, v);
        }
        spread = (mx - mn) / std::fabs(E);
        if (spread < 1e-10) break;
    }
    if (!newton(R, g, E)) return false;
    R.E = E;
    return spread <= 1e-6 && E > 0;
}

// One more zero/pole pair and two more reference points below the smallest ones.
Rat extend(const Rat& R) {
    const int k = R.k;
    std::vector<double> u(R.th.begin() + 1, R.th.begin() + 1 + k), w(R.th.begin() + 1 + k, R.th.end());
    std::sort(u.rbegin(), u.rend());
    std::sort(w.rbegin(), w.rend());
    auto ext = [](const std::vector<double>& v) {
        const size_t n = v.size();
        if (n >= 3) {
            double g1 = v[n - 2] - v[n - 1], g2 = v[n - 3] - v[n - 2];
            return v[n - 1] - (g1 + std::max(g1 - g2, 0.0));
        }
        return v[n - 1] - 3.0;
    };
    Rat S;
    S.k = k + 1;
    S.th.push_back(R.th[0]);
    for (double x : u) S.th.push_back(x);
    S.th.push_back(ext(u));
    for (double x : w) S.th.push_back(x);
    S.th.push_back(ext(w));
    const double r1 = R.T[2] / R.T[1], r2 = R.T[3] / R.T[2];
    const double n1 = R.T[1] / (r1 * r1 / r2), n0 = n1 / (r1 * r1 * r1 / (r2 * r2));
    S.T = {0.0, n0, n1};
    for (size_t i = 1; i < R.T.size(); ++i) S.T.push_back(R.T[i]);
    return S;
}

bool anchor(int k, Rat& out) {
    const double a0 = 0.5;
    Rat R;
    R.k = 1;
    R.th = {0.0, std::log(0.01), std::log(0.1)};
    R.T = {0.0, 0.01, 0.3, 1.0};
    if (!remez(R, a0)) return false;
    for (int kk = 2; kk <= k; ++kk) {
        Rat S = extend(R);
        if (!remez(S, a0)) return false;
        R = S;
    }
    out = R;
    return true;
}

// Continuation in alpha from the state R at alpha a to the requested alpha (adaptive step).
bool continue_to(Rat R, double a, double alpha, Rat& out) {
    double step = alpha > a ? 0.05 : -0.05;
    int guard = 0;
    while (a != alpha && guard++ < 10000) {
        double an = a + step;
        if ((step > 0 && an > alpha) || (step < 0 && an < alpha)) an = alpha;
        Rat S = R;
        if (!remez(S, an)) {
            step *= 0.5;
            if (std::fabs(step) < 1e-5) return false;
            continue;
        }
        R = S;
        a = an;
        step = (step > 0 ? 1 : -1) * std::min(std::fabs(step) * 1.5, 0.1);
    }
    if (a != alpha) return false;
    out = R;
    return true;
}

bool solve_bura(double alpha, int k, Rat& out) {
    Rat R;
    if (!anchor(k, R)) return false;
    return continue_to(R, 0.5, alpha, out);
}

constexpr double kGridStep = 0.05;
std::mutex g_state_mu;
std::map<std::pair<int, int>, Rat> g_states;  // (k, grid index) -> converged state at kGridStep * index

bool solve_warm(double alpha, int k, Rat& out) {
    int gi = (int)std::lround(alpha / kGridStep);
    gi = std::max(1, std::min(gi, (int)std::lround(1.0 / kGridStep) - 1));
    const double ag = kGridStep * gi;
    Rat G;
    bool have = false;
    {
        std::lock_guard<std::mutex> lk(g_state_mu);
        auto it = g_states.find({k, gi});
        if (it != g_states.end()) {
            G = it->second;
            have = true;
        }
    }
    if (!have) {
        if (!solve_bura(ag, k, G)) return solve_bura(alpha, k, out);
        std::lock_guard<std::mutex> lk(g_state_mu);
        g_states[{k, gi}] = G;
    }
    if (alpha == ag) {
        out = G;
        return true;
    }
    return continue_to(G, ag, alpha, out) || solve_bura(alpha, k, out);
}

struct Coeffs {
    std::vector<double> c, d;
    double E;
};

std::mutex g_mu;
std::map<std::pair<double, int>, Coeffs> g_cache;  // results by (alpha, k); cleared when it grows past
constexpr size_t kCacheMax = 1u << 16;             // kCacheMax entries (a continuous stream of alphas)

}  // namespace

extern "C" int bura_rational(double alpha, int k, double* c, double* d, double* E) {
    if (!(alpha > 0 && alpha < 1) || k < 1 || k > BURA_MAX_K || !c || !d) return BURA_EINVAL;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_cache.find({alpha, k});
        if (it != g_cache.end()) {
            std::memcpy(c, it->second.c.data(), sizeof(double) * (k + 1));
            std::memcpy(d, it->second.d.data(), sizeof(double) * (k + 1));
            if (E) *E = it->second.E;
            return BURA_OK;
        }
    }
    Rat R;
    if (!solve_warm(alpha, k, R)) return BURA_EREMEZ;
    // Partial fractions of t^{-1} r(t): c_0 = r(0); c_j = residue of r(t)/t at d_j = -e^{w_j}.
    std::vector<double> zu(k), zw(k);
    for (int j = 0; j < k; ++j) { zu[j] = std::exp(R.th[1 + j]); zw[j] = std::exp(R.th[1 + k + j]); }
    std::sort(zw.begin(), zw.end());  // ascending |d|: d_1 closest to 0
    Coeffs out;
    out.E = R.E;
    out.c.assign(k + 1, 0.0);
    out.d.assign(k + 1, 0.0);
    const double scale = std::exp(R.th[0]);
    double c0 = scale;
    for (int j = 0; j < k; ++j) c0 *= zu[j] / zw[j];
    out.c[0] = c0;
    for (int j = 0; j < k; ++j) {
        const double dj = -zw[j];
        double v = scale;
        for (int i = 0; i < k; ++i) {
            v *= (dj + zu[i]);
            if (i != j) v /= (dj + zw[i]);
        }
        out.c[j + 1] = v / dj;
        out.d[j + 1] = dj;
    }
    for (int j = 0; j <= k; ++j)
        if (!(out.c[j] > 0) || !std::isfinite(out.c[j])) return BURA_EREMEZ;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (g_cache.size() >= kCacheMax) g_cache.clear();
        g_cache[{alpha, k}] = out;
    }
    std::memcpy(c, out.c.data(), sizeof(double) * (k + 1));
    std::memcpy(d, out.d.data(), sizeof(double) * (k + 1));
    if (E) *E = out.E;
    return BURA_OK;
}
