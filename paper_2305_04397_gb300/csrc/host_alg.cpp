// Host-side steps of the method: task preprocessing (Sec. 2 and 3.1), the
// assignment of Algorithm 2, and the two projections of Algorithm 1.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <vector>

#include "internal.h"

namespace morap {

// --------------------------------------------------------- task preprocessing
//
// Sec. 2: a location q is a trap when no run from q reaches Q_F; Sec. 3.1:
// done_j holds on Q_F u Q_R and rho_{j+|I|}(s, q, a) = 1 exactly when q is a
// pre-sink (not accepting, every successor accepting).  A DFA is extended
// with one pre-sink when needed; here every transition into Q_F from a
// location that is not a pre-sink is routed through that added location so
// that the one-off reward is collected on every accepting run.
int preprocess_task(int32_t n_locs, int32_t q0, int32_t n_ap, const int32_t *ap_ids, const int32_t *delta,
                    const uint8_t *accepting, HostTask &T) {
    if (n_locs < 1) return fail(MORAP_EINVAL, "task: n_locs must be >= 1");
    if (n_ap < 0 || n_ap > 8) return fail(MORAP_EINVAL, "task: n_ap must be in 0..8");
    if (q0 < 0 || q0 >= n_locs) return fail(MORAP_EINVAL, "task: q0 out of range");
    if (!delta || !accepting || (n_ap > 0 && !ap_ids)) return fail(MORAP_EINVAL, "task: null array");
    const int nl = 1 << n_ap;
    std::vector<int32_t> d(delta, delta + (size_t)n_locs * nl);
    std::vector<char> acc(n_locs);
    for (int q = 0; q < n_locs; ++q) acc[q] = accepting[q] != 0;
    for (size_t k = 0; k < d.size(); ++k)
        if (d[k] < 0 || d[k] >= n_locs) return fail(MORAP_EINVAL, "task: delta target out of range");
    int first_acc = -1;
    for (int q = 0; q < n_locs; ++q) {
        if (!acc[q]) continue;
        if (first_acc < 0) first_acc = q;
        for (int w = 0; w < nl; ++w)
            if (d[(size_t)q * nl + w] != q)
                return fail(MORAP_EINVAL, "task: accepting location " + std::to_string(q) + " is not a sink");
    }
    auto leads_only_to_acc = [&](int q) {
        for (int w = 0; w < nl; ++w)
            if (!acc[d[(size_t)q * nl + w]]) return false;
        return true;
    };
    std::vector<char> presink0(n_locs);
    for (int q = 0; q < n_locs; ++q) presink0[q] = !acc[q] && leads_only_to_acc(q);
    std::vector<std::pair<int, int>> redirect;
    for (int q = 0; q < n_locs; ++q) {
        if (acc[q] || presink0[q]) continue;
        for (int w = 0; w < nl; ++w)
            if (acc[d[(size_t)q * nl + w]]) redirect.emplace_back(q, w);
    }
    int n = n_locs;
    if (!redirect.empty()) {
        const int P = n;
        d.resize((size_t)(n + 1) * nl, first_acc);
        acc.push_back(0);
        for (auto &r : redirect) d[(size_t)r.first * nl + r.second] = P;
        n += 1;
    }
    std::vector<char> pre(n), reach(n), trap(n), done(n);
    for (int q = 0; q < n; ++q) pre[q] = !acc[q] && leads_only_to_acc(q);
    for (int q = 0; q < n; ++q) reach[q] = acc[q];
    for (bool changed = true; changed;) {
        changed = false;
        for (int q = 0; q < n; ++q) {
            if (reach[q]) continue;
            for (int w = 0; w < nl; ++w)
                if (reach[d[(size_t)q * nl + w]]) {
                    reach[q] = 1;
                    changed = true;
                    break;
                }
        }
    }
    for (int q = 0; q < n; ++q) {
        trap[q] = !reach[q];
        done[q] = acc[q] || trap[q];
    }
    T = HostTask();
    T.n_locs = n;
    T.q0 = q0;
    T.n_ap = n_ap;
    T.n_letters = nl;
    T.ap_ids.assign(ap_ids, ap_ids + n_ap);
    T.delta = d;
    T.flags.resize(n);
    for (int q = 0; q < n; ++q)
        T.flags[q] = (acc[q] ? 1 : 0) | (trap[q] ? 2 : 0) | (pre[q] ? 4 : 0) | (done[q] ? 8 : 0);
    T.ploc.assign(n, -1);
    for (int pass = 0; pass < 2; ++pass)  // non-done, non-pre-sink first; pre-sinks last
        for (int q = 0; q < n; ++q)
            if (!done[q] && (pre[q] ? 1 : 0) == pass) {
                T.ploc[q] = (int)T.loc_of.size();
                T.loc_of.push_back(q);
            }
    T.n_nd = (int)T.loc_of.size();
    T.n_pre = 0;
    for (int q = 0; q < n; ++q) T.n_pre += (!done[q] && pre[q]) ? 1 : 0;
    T.nd_delta.resize((size_t)T.n_nd * nl);
    for (int pl = 0; pl < T.n_nd; ++pl)
        for (int w = 0; w < nl; ++w)
            T.nd_delta[(size_t)pl * nl + w] = (int16_t)T.ploc[d[(size_t)T.loc_of[pl] * nl + w]];
    return MORAP_OK;
}

// ----------------------------------------------------------------- assignment
//
// Algorithm 2 picks f maximising sum_j c_{f(j), j}.  This is the O(n^3)
// shortest-augmenting-path form of the Hungarian method with row and column
// potentials, run on the costs -C.
void hungarian_max(int n, const double *C, int *f) {
    const double INF = std::numeric_limits<double>::infinity();
    std::vector<double> u(n + 1, 0.0), v(n + 1, 0.0), minv(n + 1);
    std::vector<int> match(n + 1, 0), way(n + 1, 0);  // match[col] = row (1-based)
    std::vector<char> used(n + 1);
    for (int i = 1; i <= n; ++i) {
        match[0] = i;
        int j0 = 0;
        std::fill(minv.begin(), minv.end(), INF);
        std::fill(used.begin(), used.end(), 0);
        do {
            used[j0] = 1;
            const int i0 = match[j0];
            double delta = INF;
            int j1 = 0;
            for (int j = 1; j <= n; ++j) {
                if (used[j]) continue;
                const double cur = -C[(size_t)(i0 - 1) * n + (j - 1)] - u[i0] - v[j];
                if (cur < minv[j]) {
                    minv[j] = cur;
                    way[j] = j0;
                }
                if (minv[j] < delta) {
                    delta = minv[j];
                    j1 = j;
                }
            }
            for (int j = 0; j <= n; ++j) {
                if (used[j]) {
                    u[match[j]] += delta;
                    v[j] -= delta;
                } else {
                    minv[j] -= delta;
                }
            }
            j0 = j1;
        } while (match[j0] != 0);
        do {
            const int j1 = way[j0];
            match[j0] = match[j1];
            j0 = j1;
        } while (j0 != 0);
    }
    for (int j = 1; j <= n; ++j) f[j - 1] = match[j] - 1;
}

// ------------------------------------------------------------ dense QP (IPM)

// Algorithm 2's assignment for |I| agents and |J| tasks: the |I| x |J| value
// matrix is padded with zero rows (dummy agents that do nothing) or zero
// columns (dummy tasks) to a square matrix; task j goes to agent f(j), or
// to no agent (-1) when a dummy agent takes it.
void assign_tasks(int nI, int nJ, const double *C, int32_t *assign) {
    const int n = std::max(nI, nJ);
    std::vector<double> Cm((size_t)n * n, 0.0);
    for (int i = 0; i < nI; ++i)
        for (int j = 0; j < nJ; ++j) Cm[(size_t)i * n + j] = C[(size_t)i * nJ + j];
    std::vector<int> f(n);
    if (n) hungarian_max(n, Cm.data(), f.data());
    for (int j = 0; j < nJ; ++j) assign[j] = f[j] < nI ? f[j] : -1;
}

namespace {

// In-place LU with partial pivoting of a dense [n][n] matrix; returns false
// when a pivot vanishes.
bool lu_factor(int n, std::vector<double> &a, std::vector<int> &piv) {
    piv.resize(n);
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = std::fabs(a[(size_t)k * n + k]);
        for (int i = k + 1; i < n; ++i) {
            const double v = std::fabs(a[(size_t)i * n + k]);
            if (v > best) {
                best = v;
                p = i;
            }
        }
        if (best == 0.0 || !std::isfinite(best)) return false;
        piv[k] = p;
        if (p != k)
            for (int j = 0; j < n; ++j) std::swap(a[(size_t)k * n + j], a[(size_t)p * n + j]);
        const double inv = 1.0 / a[(size_t)k * n + k];
        for (int i = k + 1; i < n; ++i) {
            const double l = a[(size_t)i * n + k] * inv;
            a[(size_t)i * n + k] = l;
            if (l == 0.0) continue;
            for (int j = k + 1; j < n; ++j) a[(size_t)i * n + j] -= l * a[(size_t)k * n + j];
        }
    }
    return true;
}

// lu_factor swaps whole rows (multipliers included), so P A = L U with P the
// product of the swaps in order: apply P to b first, then substitute.
void lu_solve(int n, const std::vector<double> &a, const std::vector<int> &piv, double *b) {
    for (int k = 0; k < n; ++k)
        if (piv[k] != k) std::swap(b[k], b[piv[k]]);
    for (int k = 0; k < n; ++k)
        for (int i = k + 1; i < n; ++i) b[i] -= a[(size_t)i * n + k] * b[k];
    for (int k = n - 1; k >= 0; --k) {
        double s = b[k];
        for (int j = k + 1; j < n; ++j) s -= a[(size_t)k * n + j] * b[j];
        b[k] = s / a[(size_t)k * n + k];
    }
}

double inf_norm(const std::vector<double> &v) {
    double m = 0.0;
    for (double e : v) m = std::max(m, std::fabs(e));
    return m;
}

}  // namespace

// Solve the QP with the inequalities in `act` held as equalities (the KKT
// system of the equality-constrained problem).  Accepts the point only if it
// is feasible for every inequality and the multipliers of the held ones are
// nonnegative, i.e. it is the exact optimum for that active set.
bool qp_active_set_solve(int n, const double *G, const double *c, int m, const double *A, const double *b, int p,
                         const double *E, const double *d, const std::vector<int> &act, double scale,
                         double *x_out) {
    const int na = (int)act.size(), N = n + na + p;
    std::vector<double> K((size_t)N * N, 0.0), r(N, 0.0);
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) K[(size_t)i * N + j] = G[(size_t)i * n + j];
        r[i] = -c[i];
    }
    for (int q = 0; q < na; ++q) {
        const double *ak = A + (size_t)act[q] * n;
        for (int j = 0; j < n; ++j) {
            K[(size_t)(n + q) * N + j] = ak[j];
            K[(size_t)j * N + (n + q)] = ak[j];
        }
        r[n + q] = b[act[q]];
    }
    for (int q = 0; q < p; ++q) {
        for (int j = 0; j < n; ++j) {
            K[(size_t)(n + na + q) * N + j] = E[(size_t)q * n + j];
            K[(size_t)j * N + (n + na + q)] = E[(size_t)q * n + j];
        }
        r[n + na + q] = d[q];
    }
    std::vector<int> piv;
    if (!lu_factor(N, K, piv)) return false;
    lu_solve(N, K, piv, r.data());
    const double ftol = 1e-12 * scale;
    for (int q = 0; q < na; ++q)
        if (r[n + q] < -ftol) return false;  // a held constraint wants to be released
    for (int k = 0; k < m; ++k) {
        double ax = 0.0;
        for (int j = 0; j < n; ++j) ax += A[(size_t)k * n + j] * r[j];
        if (ax > b[k] + ftol) return false;
    }
    std::copy(r.begin(), r.begin() + n, x_out);
    return true;
}

int qp_solve(int n, const double *G, const double *c, int m, const double *A, const double *b, int p,
             const double *E, const double *d, double *x, double tol, int max_iter) {
    std::vector<double> s(m), z(m, 1.0), y(p, 0.0);
    std::vector<double> rd(n), rp(m), re(p), K((size_t)(n + p) * (n + p)), rhs(n + p);
    std::vector<double> dx(n), ds(m), dz(m), dy(p), dxa(n), dsa(m), dza(m), dya(p), rc(m), Ax(m);
    std::vector<int> piv;
    double scale = 1.0;
    for (int i = 0; i < n; ++i) scale = std::max(scale, std::fabs(c[i]));
    for (int i = 0; i < m; ++i) scale = std::max(scale, std::fabs(b[i]));
    for (int i = 0; i < m; ++i) {
        double ax = 0.0;
        for (int j = 0; j < n; ++j) ax += A[(size_t)i * n + j] * x[j];
        s[i] = std::max(b[i] - ax, 1.0);
    }
    auto residuals = [&]() {
        for (int i = 0; i < n; ++i) {
            double acc = c[i];
            for (int j = 0; j < n; ++j) acc += G[(size_t)i * n + j] * x[j];
            rd[i] = acc;
        }
        for (int k = 0; k < m; ++k) {
            double ax = 0.0;
            for (int j = 0; j < n; ++j) ax += A[(size_t)k * n + j] * x[j];
            Ax[k] = ax;
            rp[k] = ax + s[k] - b[k];
            for (int j = 0; j < n; ++j) rd[j] += A[(size_t)k * n + j] * z[k];
        }
        for (int k = 0; k < p; ++k) {
            double ex = 0.0;
            for (int j = 0; j < n; ++j) ex += E[(size_t)k * n + j] * x[j];
            re[k] = ex - d[k];
            for (int j = 0; j < n; ++j) rd[j] += E[(size_t)k * n + j] * y[k];
        }
    };
    // Newton direction for complementarity residual rc (s.z + ... = 0 target).
    auto direction = [&](const std::vector<double> &rcv, std::vector<double> &ox, std::vector<double> &os,
                         std::vector<double> &oz, std::vector<double> &oy) {
        for (int i = 0; i < n; ++i) rhs[i] = -rd[i];
        for (int k = 0; k < m; ++k) {
            const double g = (-rcv[k] + z[k] * rp[k]) / s[k];
            for (int j = 0; j < n; ++j) rhs[j] -= A[(size_t)k * n + j] * g;
        }
        for (int k = 0; k < p; ++k) rhs[n + k] = -re[k];
        std::vector<double> sol(rhs);
        lu_solve(n + p, K, piv, sol.data());
        for (int i = 0; i < n; ++i) ox[i] = sol[i];
        for (int k = 0; k < p; ++k) oy[k] = sol[n + k];
        for (int k = 0; k < m; ++k) {
            double adx = 0.0;
            for (int j = 0; j < n; ++j) adx += A[(size_t)k * n + j] * ox[j];
            os[k] = -rp[k] - adx;
            oz[k] = (-rcv[k] + z[k] * rp[k] + z[k] * adx) / s[k];
        }
    };
    auto max_step = [&](const std::vector<double> &ds_, const std::vector<double> &dz_) {
        double a = 1.0;
        for (int k = 0; k < m; ++k) {
            if (ds_[k] < 0) a = std::min(a, -s[k] / ds_[k]);
            if (dz_[k] < 0) a = std::min(a, -z[k] / dz_[k]);
        }
        return a;
    };
    for (int it = 0; it < max_iter; ++it) {
        residuals();
        const double mu = m > 0 ? [&] {
            double acc = 0.0;
            for (int k = 0; k < m; ++k) acc += s[k] * z[k];
            return acc / m;
        }()
                                : 0.0;
        const double res = std::max(inf_norm(rd), std::max(inf_norm(rp), inf_norm(re)));
        if (res <= tol * scale && mu <= 1e-3 * tol * scale) return 0;
        // Near the optimum the active constraints are those whose slack has
        // gone to zero while the multiplier has not: solve for them exactly
        // (an interior point's x is only accurate to the square root of the
        // duality gap, and the gap cannot shrink much below rounding).
        if (m > 0 && res <= 1e-7 * scale && mu <= 1e-6 * scale) {
            std::vector<int> act;
            for (int k = 0; k < m; ++k)
                if (z[k] > s[k]) act.push_back(k);
            if (qp_active_set_solve(n, G, c, m, A, b, p, E, d, act, scale, x)) return 0;
        }
        // K = [G + A' diag(z/s) A, E'; E, 0]
        std::fill(K.begin(), K.end(), 0.0);
        const int N = n + p;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) K[(size_t)i * N + j] = G[(size_t)i * n + j];
        for (int k = 0; k < m; ++k) {
            const double w = z[k] / s[k];
            const double *ak = A + (size_t)k * n;
            for (int i = 0; i < n; ++i) {
                if (ak[i] == 0.0) continue;
                const double wi = w * ak[i];
                for (int j = 0; j < n; ++j) K[(size_t)i * N + j] += wi * ak[j];
            }
        }
        for (int k = 0; k < p; ++k)
            for (int j = 0; j < n; ++j) {
                K[(size_t)(n + k) * N + j] = E[(size_t)k * n + j];
                K[(size_t)j * N + (n + k)] = E[(size_t)k * n + j];
            }
        if (!lu_factor(N, K, piv)) return 2;
        // predictor
        for (int k = 0; k < m; ++k) rc[k] = s[k] * z[k];
        direction(rc, dxa, dsa, dza, dya);
        const double aa = max_step(dsa, dza);
        double mu_aff = 0.0;
        for (int k = 0; k < m; ++k) mu_aff += (s[k] + aa * dsa[k]) * (z[k] + aa * dza[k]);
        mu_aff = m > 0 ? mu_aff / m : 0.0;
        const double sigma = mu > 0 ? std::pow(mu_aff / mu, 3.0) : 0.0;
        // corrector
        for (int k = 0; k < m; ++k) rc[k] = s[k] * z[k] + dsa[k] * dza[k] - sigma * mu;
        direction(rc, dx, ds, dz, dy);
        const double a = std::min(1.0, 0.995 * max_step(ds, dz));
        for (int i = 0; i < n; ++i) x[i] += a * dx[i];
        for (int k = 0; k < m; ++k) {
            s[k] = std::max(s[k] + a * ds[k], 1e-300);
            z[k] = std::max(z[k] + a * dz[k], 1e-300);
        }
        for (int k = 0; k < p; ++k) y[k] += a * dy[k];
    }
    return 1;
}

// Algorithm 1, outer bound: argmin_z ||t - z||_M  s.t.  w'.z <= w'.r' for all
// (w', r') in Lambda.
int project_halfspaces(int n, int m, const double *t, const double *A, const double *b, const double *M,
                       double *z) {
    bool inside = true;
    for (int k = 0; k < m && inside; ++k) {
        double at = 0.0;
        for (int j = 0; j < n; ++j) at += A[(size_t)k * n + j] * t[j];
        if (at > b[k]) inside = false;
    }
    std::copy(t, t + n, z);
    if (inside) return 0;
    std::vector<double> G((size_t)n * n), c(n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) G[(size_t)i * n + j] = M ? M[(size_t)i * n + j] : (i == j ? 1.0 : 0.0);
    for (int i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int j = 0; j < n; ++j) acc += G[(size_t)i * n + j] * t[j];
        c[i] = -acc;
    }
    return qp_solve(n, G.data(), c.data(), m, A, b, 0, nullptr, nullptr, z);
}

// Algorithm 1, inner bound: argmin_x ||t - x||_M over x <= sum_l lam_l Phi_l,
// lam >= 0, sum lam = 1 (variables x and lam).
int project_down_hull(int n, int m, const double *t, const double *Phi, const double *M, double *x, double *lambda) {
    const int N = n + m;
    std::vector<double> G((size_t)N * N, 0.0), c(N, 0.0), v(N, 0.0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) G[(size_t)i * N + j] = M ? M[(size_t)i * n + j] : (i == j ? 1.0 : 0.0);
    for (int i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int j = 0; j < n; ++j) acc += G[(size_t)i * N + j] * t[j];
        c[i] = -acc;
    }
    const int mi = n + m;
    std::vector<double> A((size_t)mi * N, 0.0), b(mi, 0.0), E(N, 0.0), d(1, 1.0);
    for (int k = 0; k < n; ++k) {
        A[(size_t)k * N + k] = 1.0;
        for (int l = 0; l < m; ++l) A[(size_t)k * N + n + l] = -Phi[(size_t)l * n + k];
    }
    for (int l = 0; l < m; ++l) A[(size_t)(n + l) * N + n + l] = -1.0;
    for (int l = 0; l < m; ++l) E[n + l] = 1.0;
    for (int l = 0; l < m; ++l) v[n + l] = 1.0 / m;
    for (int i = 0; i < n; ++i) {
        double hull = 0.0;
        for (int l = 0; l < m; ++l) hull += Phi[(size_t)l * n + i] / m;
        v[i] = std::min(t[i], hull) - 1.0;
    }
    const int rc = qp_solve(N, G.data(), c.data(), mi, A.data(), b.data(), 1, E.data(), d.data(), v.data());
    // With a diagonal metric the projection never exceeds t in any objective
    // (x_i = min(t_i, (Phi' lam)_i)), so clipping removes only roundoff; with a
    // general metric it may exceed t and is returned as solved.
    bool diagonal = true;
    for (int i = 0; M && i < n; ++i)
        for (int j = 0; j < n; ++j)
            if (i != j && M[(size_t)i * n + j] != 0.0) diagonal = false;
    for (int i = 0; i < n; ++i) x[i] = diagonal ? std::min(v[i], t[i]) : v[i];
    if (lambda) {
        // the convex weights, cleaned of the solver's roundoff (>= 0, sum 1)
        double sum = 0.0;
        for (int l = 0; l < m; ++l) sum += (lambda[l] = std::max(v[n + l], 0.0));
        for (int l = 0; l < m; ++l) lambda[l] = sum > 0.0 ? lambda[l] / sum : 1.0 / m;
    }
    return rc;
}

// ------------------------------------------------------------- Algorithm 1

double mnorm(int n, const double *v, const double *M) {
    double acc = 0.0;
    for (int i = 0; i < n; ++i) {
        double mv = 0.0;
        for (int j = 0; j < n; ++j) mv += (M ? M[(size_t)i * n + j] : (i == j ? 1.0 : 0.0)) * v[j];
        acc += v[i] * mv;
    }
    return std::sqrt(std::max(acc, 0.0));
}

void Alg1::init(int n_obj, const double *t_in, const double *M_in, double eps_in, int max_iter_in,
                bool verify_only_in) {
    verify_only = verify_only_in;
    decided = false;
    n = n_obj;
    t.assign(t_in, t_in + n);
    if (M_in)
        M.assign(M_in, M_in + (size_t)n * n);
    else
        M.clear();
    w.assign(n, 0.0);
    w[0] = 1.0;  // the first direction is e_1
    t_dn = t;
    t_up.assign(n, -HUGE_VAL);
    Phi.clear();
    A.clear();
    b.clear();
    w_hist.clear();
    r_hist.clear();
    f_hist.clear();
    lambda.clear();
    moved = false;
    done = false;
    it = 0;
    status = 0;
    dist = HUGE_VAL;
    eps = eps_in;
    max_iter = max_iter_in;
}

// One pass of the loop body with the supporting point r for direction w:
// the point joins Phi and the halfspace {z : w.z <= w.r} joins Lambda; the
// outer bound moves when w.r < w.t_down; the inner bound is re-projected;
// then the loop test on ||t_down - t_up||_M, and the next direction
// w = M (t - t_up) / ||M (t - t_up)||_1.
void Alg1::step(const double *r, const int32_t *assign, int n_tasks) {
    const double *Mp = M.empty() ? nullptr : M.data();
    w_hist.insert(w_hist.end(), w.begin(), w.end());
    r_hist.insert(r_hist.end(), r, r + n);
    if (assign && n_tasks > 0) {
        f_tasks = n_tasks;
        f_hist.insert(f_hist.end(), assign, assign + n_tasks);
    }
    ++it;
    Phi.insert(Phi.end(), r, r + n);
    A.insert(A.end(), w.begin(), w.end());
    double wr = 0.0, wt = 0.0;
    for (int i = 0; i < n; ++i) {
        wr += w[i] * r[i];
        wt += w[i] * t_dn[i];
    }
    b.push_back(wr);
    if (wr < wt) {
        moved = true;
        if (verify_only) {
            // the paper's verification-only loop breaks here, before the
            // outer bound is projected: t is separated from the achievable set
            decided = true;
            done = true;
            return;
        }
        project_halfspaces(n, (int)b.size(), t.data(), A.data(), b.data(), Mp, t_dn.data());
    }
    lambda.assign(it, 0.0);
    project_down_hull(n, it, t.data(), Phi.data(), Mp, t_up.data(), lambda.data());
    std::vector<double> d(n);
    for (int i = 0; i < n; ++i) d[i] = t_dn[i] - t_up[i];
    dist = mnorm(n, d.data(), Mp);
    if (dist <= eps || it >= max_iter) {
        done = true;
        return;
    }
    double l1 = 0.0;
    for (int i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int j = 0; j < n; ++j) acc += (Mp ? Mp[(size_t)i * n + j] : (i == j ? 1.0 : 0.0)) * (t[j] - t_up[j]);
        d[i] = acc;
        l1 += std::fabs(acc);
    }
    if (!(l1 > 0.0)) {  // t_up == t: t is achievable, nothing left to separate
        done = true;
        return;
    }
    for (int i = 0; i < n; ++i) w[i] = std::max(d[i], 0.0) / l1;
}

int alg1_result(const Alg1 &q, morap_point_result *res) {
    int status = q.status;
    const bool converged = q.dist <= q.eps || q.decided;
    if (!converged && status == MORAP_OK) status = MORAP_ENOTCONV;
    res->feasible = q.moved ? 0 : 1;
    res->iterations = q.it;
    res->converged = converged ? 1 : 0;
    res->status = status;
    res->distance = q.dist;
    if (res->t_up) std::copy(q.t_up.begin(), q.t_up.end(), res->t_up);
    if (res->t_down) std::copy(q.t_dn.begin(), q.t_dn.end(), res->t_down);
    if (res->w_hist) std::copy(q.w_hist.begin(), q.w_hist.end(), res->w_hist);
    if (res->r_hist) std::copy(q.r_hist.begin(), q.r_hist.end(), res->r_hist);
    if (res->lambda) std::copy(q.lambda.begin(), q.lambda.end(), res->lambda);
    if (res->assign_hist && !q.f_hist.empty()) std::copy(q.f_hist.begin(), q.f_hist.end(), res->assign_hist);
    return status;
}

}  // namespace morap
