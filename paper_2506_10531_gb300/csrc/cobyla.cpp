// cobyla.cpp -- derivative-free minimisation for the gradient-free outer loop of Section IV (the
// paper tunes each sub-QUBO's angles with COBYLA). Written from the method's published
// description (M. J. D. Powell, "A direct search optimization method that models the objective
// and constraint functions by linear interpolation", Advances in Optimization and Numerical
// Analysis, 1994), unconstrained case:
//   * the n+1 vertices of a simplex carry function values; the linear function interpolating
//     them is the model, its gradient g solves A g = f_j - f_opt, where the rows of A are the
//     vertices' offsets from the best vertex;
//   * a trust-region step moves the best vertex by rho against g (the model's minimiser on the
//     ball of radius rho) and replaces the vertex whose exchange keeps the simplex volume largest
//     (|det| ratio = |d . b_r|, b_r the r-th column of A^-1), favouring far vertices;
//   * when a vertex lies farther than beta rho from the best one, or closer than alpha rho to the
//     face opposite it (that distance is 1 / |b_r|), a geometry step replaces it by the best
//     vertex plus gamma rho along b_r;
//   * a step that achieves less than a tenth of the predicted reduction halves rho, down to
//     rho_end, where the method stops.
// The interface is reverse communication (ask a point, tell its value), so that a caller can
// evaluate the points of many independent minimisations in one batched launch.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/qaoa.h"
#include "qaoa_host.h"

namespace {

constexpr double kAlpha = 0.25;   // minimum distance of a vertex from its opposite face / rho
constexpr double kBeta = 2.1;     // maximum distance of a vertex from the best vertex / rho
constexpr double kGamma = 0.5;    // length of a geometry step / rho
constexpr double kDelta = 1.1;    // distance weight in the choice of the vertex to replace

}  // namespace

struct qaoa_cobyla {
    int n = 0;
    double rho = 0.0, rho_end = 0.0;
    int maxfun = 0, nfev = 0;
    std::vector<double> V;        // (n + 1) x n vertices
    std::vector<double> F;        // n + 1 values
    std::vector<int> pending;     // vertices still to evaluate (initial or rebuilt simplex)
    int phase = 0;                // 0: evaluating `pending`, 1: a trial point is out, 2: done
    std::vector<double> trial;
    int trial_kind = 0;           // 0: trust-region step, 1: geometry step replacing geo_j
    int geo_j = -1;
    double pred = 0.0;            // predicted reduction of the trust-region step
    bool poor = false;            // the last trust-region step achieved too little
    int opt = 0;
    std::vector<int> rows;        // vertex of each row of A
    std::vector<double> A, B, g;  // offsets, their inverse, model gradient
};

namespace {

double* vert(qaoa_cobyla* s, int j) { return s->V.data() + (size_t)j * s->n; }

// Gauss-Jordan inverse with partial pivoting; false when a pivot is negligible.
bool invert(int n, const std::vector<double>& M, std::vector<double>& inv) {
    std::vector<double> a(M);
    inv.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
    double scale = 0.0;
    for (double v : a) scale = std::max(scale, std::fabs(v));
    if (!(scale > 0.0)) return false;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(a[(size_t)r * n + c]) > std::fabs(a[(size_t)piv * n + c])) piv = r;
        const double pv = a[(size_t)piv * n + c];
        if (!(std::fabs(pv) > 1e-13 * scale)) return false;
        if (piv != c)
            for (int k = 0; k < n; ++k) {
                std::swap(a[(size_t)piv * n + k], a[(size_t)c * n + k]);
                std::swap(inv[(size_t)piv * n + k], inv[(size_t)c * n + k]);
            }
        for (int k = 0; k < n; ++k) {
            a[(size_t)c * n + k] /= pv;
            inv[(size_t)c * n + k] /= pv;
        }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const double f = a[(size_t)r * n + c];
            if (f == 0.0) continue;
            for (int k = 0; k < n; ++k) {
                a[(size_t)r * n + k] -= f * a[(size_t)c * n + k];
                inv[(size_t)r * n + k] -= f * inv[(size_t)c * n + k];
            }
        }
    }
    return true;
}

void shrink(qaoa_cobyla* s) {
    if (s->rho <= s->rho_end) {
        s->phase = 2;
        return;
    }
    s->rho = (0.5 * s->rho > 1.5 * s->rho_end) ? 0.5 * s->rho : s->rho_end;
}

// Rebuild the simplex around the best vertex with coordinate offsets rho (degenerate simplex).
void rebuild(qaoa_cobyla* s) {
    const int n = s->n;
    s->pending.clear();
    int r = 0;
    for (int j = 0; j <= n; ++j) {
        if (j == s->opt) continue;
        double* v = vert(s, j);
        std::memcpy(v, vert(s, s->opt), sizeof(double) * n);
        v[r++] += s->rho;
        s->F[j] = HUGE_VAL;
        s->pending.push_back(j);
    }
    s->phase = 0;
}

// Choose the next point to evaluate (or finish).
void plan_next(qaoa_cobyla* s) {
    const int n = s->n;
    for (;;) {
        if (s->phase == 2) return;
        if (s->nfev >= s->maxfun) {
            s->phase = 2;
            return;
        }
        s->opt = 0;
        for (int j = 1; j <= n; ++j)
            if (s->F[j] < s->F[s->opt]) s->opt = j;
        if (!(s->F[s->opt] < HUGE_VAL)) {   // no finite value anywhere: nothing to model
            s->phase = 2;
            return;
        }
        // a vertex whose value was not finite cannot enter the linear model: move it halfway
        // towards the best vertex and evaluate it again (a geometry step of half its length)
        for (int j = 0; j <= n; ++j) {
            if (j == s->opt || s->F[j] < HUGE_VAL) continue;
            const double* xo = vert(s, s->opt);
            const double* v = vert(s, j);
            s->trial.assign(n, 0.0);
            for (int k = 0; k < n; ++k) s->trial[k] = xo[k] + 0.5 * (v[k] - xo[k]);
            s->trial_kind = 1;
            s->geo_j = j;
            s->phase = 1;
            return;
        }
        s->rows.clear();
        for (int j = 0; j <= n; ++j)
            if (j != s->opt) s->rows.push_back(j);
        s->A.assign((size_t)n * n, 0.0);
        const double* xo = vert(s, s->opt);
        for (int r = 0; r < n; ++r) {
            const double* v = vert(s, s->rows[r]);
            for (int k = 0; k < n; ++k) s->A[(size_t)r * n + k] = v[k] - xo[k];
        }
        if (!invert(n, s->A, s->B)) {
            rebuild(s);
            return;
        }
        // g = B df (A g = df)
        s->g.assign(n, 0.0);
        for (int r = 0; r < n; ++r) {
            const double df = s->F[s->rows[r]] - s->F[s->opt];
            for (int k = 0; k < n; ++k) s->g[k] += s->B[(size_t)k * n + r] * df;
        }
        // acceptability: eta_r = |row r of A|, sigma_r = 1 / |column r of B|
        int far = -1, flat = -1;
        double eta_max = 0.0, sig_min = 0.0;
        for (int r = 0; r < n; ++r) {
            double e = 0.0, b = 0.0;
            for (int k = 0; k < n; ++k) {
                e += s->A[(size_t)r * n + k] * s->A[(size_t)r * n + k];
                b += s->B[(size_t)k * n + r] * s->B[(size_t)k * n + r];
            }
            e = std::sqrt(e);
            const double sig = 1.0 / std::sqrt(b);
            if (far < 0 || e > eta_max) { far = r; eta_max = e; }
            if (flat < 0 || sig < sig_min) { flat = r; sig_min = sig; }
        }
        int geo = -1;
        if (eta_max > kBeta * s->rho) geo = far;
        else if (sig_min < kAlpha * s->rho) geo = flat;
        if (geo < 0 && s->poor) {
            // a poor step from an acceptable simplex: the model is good only on a smaller scale
            s->poor = false;
            shrink(s);
            continue;
        }
        s->trial.assign(n, 0.0);
        if (geo >= 0) {
            double bn = 0.0, gb = 0.0;
            for (int k = 0; k < n; ++k) {
                const double b = s->B[(size_t)k * n + geo];
                bn += b * b;
                gb += s->g[k] * b;
            }
            bn = std::sqrt(bn);
            const double sign = gb > 0.0 ? -1.0 : 1.0;
            for (int k = 0; k < n; ++k) s->trial[k] = xo[k] + sign * kGamma * s->rho * s->B[(size_t)k * n + geo] / bn;
            s->trial_kind = 1;
            s->geo_j = s->rows[geo];
            s->phase = 1;
            return;
        }
        double gn = 0.0;
        for (int k = 0; k < n; ++k) gn += s->g[k] * s->g[k];
        gn = std::sqrt(gn);
        if (!(gn > 0.0) || !std::isfinite(gn)) {   // flat model: a smaller radius, or the end
            shrink(s);
            continue;
        }
        for (int k = 0; k < n; ++k) s->trial[k] = xo[k] - s->rho * s->g[k] / gn;
        s->pred = s->rho * gn;
        s->trial_kind = 0;
        s->phase = 1;
        return;
    }
}

}  // namespace

extern "C" qaoa_status qaoa_cobyla_create(int nvar, const double* x0, double rhobeg, double rhoend,
                                          int maxfun, qaoa_cobyla** out) {
    if (!out || !x0 || nvar < 1 || nvar > 256 || !(rhobeg > 0.0) || !(rhoend > 0.0) || rhoend > rhobeg ||
        maxfun < nvar + 2)
        return qaoa::set_error(QAOA_E_INVALID, "cobyla_create: bad arguments");
    qaoa_cobyla* s = new qaoa_cobyla();
    s->n = nvar;
    s->rho = rhobeg;
    s->rho_end = rhoend;
    s->maxfun = maxfun;
    s->V.assign((size_t)(nvar + 1) * nvar, 0.0);
    s->F.assign(nvar + 1, HUGE_VAL);   // not evaluated yet
    for (int j = 0; j <= nvar; ++j) {
        std::memcpy(vert(s, j), x0, sizeof(double) * nvar);
        if (j > 0) vert(s, j)[j - 1] += rhobeg;
        s->pending.push_back(j);
    }
    s->phase = 0;
    *out = s;
    return QAOA_OK;
}

extern "C" int qaoa_cobyla_ask(qaoa_cobyla* s, double* x) {
    if (!s || !x) return 0;
    if (s->phase == 0) {
        std::memcpy(x, vert(s, s->pending.back()), sizeof(double) * s->n);
        return 1;
    }
    if (s->phase == 1) {
        std::memcpy(x, s->trial.data(), sizeof(double) * s->n);
        return 1;
    }
    int best = 0;
    for (int j = 1; j <= s->n; ++j)
        if (s->F[j] < s->F[best]) best = j;
    std::memcpy(x, vert(s, best), sizeof(double) * s->n);
    return 0;
}

extern "C" qaoa_status qaoa_cobyla_tell(qaoa_cobyla* s, double f) {
    if (!s) return qaoa::set_error(QAOA_E_INVALID, "cobyla_tell: NULL state");
    if (s->phase == 2) return qaoa::set_error(QAOA_E_INVALID, "cobyla_tell: the minimisation has finished");
    if (!std::isfinite(f)) f = HUGE_VAL;
    ++s->nfev;
    if (s->phase == 0) {
        s->F[s->pending.back()] = f;
        s->pending.pop_back();
        if (s->pending.empty()) plan_next(s);
        else if (s->nfev >= s->maxfun) s->phase = 2;
        return QAOA_OK;
    }
    const int n = s->n;
    if (s->trial_kind == 1) {
        std::memcpy(vert(s, s->geo_j), s->trial.data(), sizeof(double) * n);
        s->F[s->geo_j] = f;
        plan_next(s);
        return QAOA_OK;
    }
    // a trust-region trial without a finite value stays out of the simplex: treated as a poor
    // step, it leads to a smaller radius (after a geometry repair if one is due)
    if (!(f < HUGE_VAL)) {
        s->poor = true;
        plan_next(s);
        return QAOA_OK;
    }
    // trust-region step: the trial replaces the vertex that keeps the simplex volume largest,
    // far vertices weighted up
    const double fopt = s->F[s->opt];
    const double* xo = vert(s, s->opt);
    int rep = -1;
    double best = -1.0;
    for (int r = 0; r < n; ++r) {
        double db = 0.0, e = 0.0;
        for (int k = 0; k < n; ++k) {
            db += (s->trial[k] - xo[k]) * s->B[(size_t)k * n + r];
            e += s->A[(size_t)r * n + k] * s->A[(size_t)r * n + k];
        }
        const double score = std::fabs(db) * std::max(1.0, std::sqrt(e) / (kDelta * s->rho));
        if (score > best) { best = score; rep = r; }
    }
    const int j = s->rows[rep];
    std::memcpy(vert(s, j), s->trial.data(), sizeof(double) * n);
    s->F[j] = f;
    const double ratio = (fopt - f) / s->pred;
    // a poor step first repairs the simplex geometry (if needed), then halves rho
    s->poor = !(ratio >= 0.1);
    plan_next(s);
    return QAOA_OK;
}

extern "C" qaoa_status qaoa_cobyla_result(qaoa_cobyla* s, double* x, double* f, int* nfev) {
    if (!s) return qaoa::set_error(QAOA_E_INVALID, "cobyla_result: NULL state");
    int best = 0;
    for (int j = 1; j <= s->n; ++j)
        if (s->F[j] < s->F[best]) best = j;
    if (x) std::memcpy(x, vert(s, best), sizeof(double) * s->n);
    if (f) *f = s->F[best];
    if (nfev) *nfev = s->nfev;
    return QAOA_OK;
}

extern "C" void qaoa_cobyla_destroy(qaoa_cobyla* s) { delete s; }
