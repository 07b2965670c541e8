// 1-D nodal tables (host, FP64): Legendre-Gauss-Lobatto collocation points and
// Lagrange polynomials (Sec. II.A.3), Gauss-Legendre quadrature (Sec. II.A.5),
// and the interpolation / derivative operators of Sec. II.F.4 for every degree
// pair, including half-interval (2:1 mortar and child) interpolation.
#include <cmath>
#include <vector>

#include "internal.h"

namespace dg {
namespace {

// Legendre P_N(x) and its first two derivatives by the three-term recurrence.
void legendre(int N, double x, double& P, double& dP, double& d2P) {
    double p0 = 1.0, p1 = x;
    if (N == 0) { P = 1.0; dP = 0.0; d2P = 0.0; return; }
    for (int k = 2; k <= N; ++k) {
        double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
    }
    P = p1;
    // derivatives from the Legendre ODE (valid for |x| < 1)
    double pm1 = p0;  // P_{N-1}
    dP = N * (x * P - pm1) / (x * x - 1.0);
    d2P = (2.0 * x * dP - N * (N + 1.0) * P) / (1.0 - x * x);
}

void lgl(int n, std::vector<double>& x, std::vector<double>& w) {
    const int N = n - 1;
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    x[0] = -1.0;
    x[N] = 1.0;
    for (int i = 1; i < N; ++i) {
        // Chebyshev-Gauss-Lobatto initial guess, Newton on P_N'
        double t = -std::cos(M_PI * i / N);
        for (int it = 0; it < 100; ++it) {
            double P, dP, d2P;
            legendre(N, t, P, dP, d2P);
            double dt = dP / d2P;
            t -= dt;
            if (std::fabs(dt) < 1e-16) break;
        }
        x[i] = t;
    }
    for (int i = 0; i <= N; ++i) {
        double P, dP, d2P;
        if (i == 0 || i == N) {
            P = (i == 0 && (N % 2)) ? -1.0 : 1.0;
        } else {
            legendre(N, x[i], P, dP, d2P);
        }
        w[i] = 2.0 / (N * (N + 1.0) * P * P);
    }
}

void gl(int q, std::vector<double>& x, std::vector<double>& w) {
    x.assign(q, 0.0);
    w.assign(q, 0.0);
    for (int i = 0; i < q; ++i) {
        double t = -std::cos(M_PI * (i + 0.75) / (q + 0.5));
        double P, dP, d2P;
        for (int it = 0; it < 100; ++it) {
            legendre(q, t, P, dP, d2P);
            double dt = P / dP;
            t -= dt;
            if (std::fabs(dt) < 1e-16) break;
        }
        legendre(q, t, P, dP, d2P);
        x[i] = t;
        w[i] = 2.0 / ((1.0 - t * t) * dP * dP);
    }
}

double lag(const std::vector<double>& nodes, int a, double t) {
    double v = 1.0;
    for (size_t m = 0; m < nodes.size(); ++m)
        if ((int)m != a) v *= (t - nodes[m]) / (nodes[a] - nodes[m]);
    return v;
}

double dlag(const std::vector<double>& nodes, int a, double t) {
    double s = 0.0;
    const int n = (int)nodes.size();
    for (int m = 0; m < n; ++m) {
        if (m == a) continue;
        double term = 1.0 / (nodes[a] - nodes[m]);
        for (int k = 0; k < n; ++k)
            if (k != a && k != m) term *= (t - nodes[k]) / (nodes[a] - nodes[k]);
        s += term;
    }
    return s;
}

double sub(int pos, double s) { return pos == 0 ? s : (pos == 1 ? 0.5 * (s - 1.0) : 0.5 * (s + 1.0)); }

}  // namespace

void build_tables(std::vector<double>& tab) {
    tab.assign((size_t)TabIndex::Count * kTabStride, 0.0);
    std::vector<double> xl[kMaxN + 1], wl[kMaxN + 1], xg[kMaxN + 1], wg[kMaxN + 1];
    for (int n = kMinN; n <= kMaxN; ++n) {
        lgl(n, xl[n], wl[n]);
        gl(n, xg[n], wg[n]);
    }
    for (int n = kMinN; n <= kMaxN; ++n) {
        double* I = &tab[tab_n(TabIndex::I, n)];
        double* Dg = &tab[tab_n(TabIndex::Dg, n)];
        double* DL = &tab[tab_n(TabIndex::DL, n)];
        double* IDg = &tab[tab_n(TabIndex::IDg, n)];
        for (int i = 0; i < n; ++i)
            for (int a = 0; a < n; ++a) {
                I[i * n + a] = lag(xl[n], a, xg[n][i]);
                Dg[i * n + a] = dlag(xg[n], a, xg[n][i]);
                DL[i * n + a] = dlag(xl[n], a, xl[n][i]);
                IDg[i * n + a] = dlag(xl[n], a, xg[n][i]);
            }
        for (int i = 0; i < n; ++i) {
            tab[tab_n(TabIndex::LGLx, n) + i] = xl[n][i];
            tab[tab_n(TabIndex::GLx, n) + i] = xg[n][i];
            tab[tab_n(TabIndex::GLw, n) + i] = wg[n][i];
        }
        for (int q = kMinN; q <= kMaxN; ++q)
            for (int pos = 0; pos < 3; ++pos) {
                double* Im = &tab[tab_m(TabIndex::Im, n, q, pos)];
                double* Dm = &tab[tab_m(TabIndex::Dm, n, q, pos)];
                for (int i = 0; i < q; ++i)
                    for (int a = 0; a < n; ++a) {
                        double t = sub(pos, xg[q][i]);
                        Im[i * n + a] = lag(xl[n], a, t);
                        Dm[i * n + a] = dlag(xl[n], a, t);
                    }
            }
    }
    for (int nH = kMinN; nH <= kMaxN; ++nH)
        for (int nh = kMinN; nh <= kMaxN; ++nh)
            for (int b = 0; b < 2; ++b) {
                double* C = &tab[tab_ci(nH, nh, b)];
                for (int i = 0; i < nh; ++i)
                    for (int a = 0; a < nH; ++a) C[i * nH + a] = lag(xl[nH], a, 0.5 * (xl[nh][i] + 2.0 * b - 1.0));
            }
}

void build_face_tables(const std::vector<double>& tab, std::vector<double>& ftab, FaceTabs& ft) {
    ftab.clear();
    for (int n = kMinN; n <= kMaxN; ++n)
        for (int q = kMinN; q <= kMaxN; ++q)
            for (int pos = 0; pos < 3; ++pos) {
                if (q < n) {
                    ft.off[n - kMinN][q - kMinN][pos] = -1;
                    continue;
                }
                ft.off[n - kMinN][q - kMinN][pos] = (int)ftab.size();   // even: pairs stay aligned
                const double* Im = &tab[tab_m(TabIndex::Im, n, q, pos)];
                const double* Dm = &tab[tab_m(TabIndex::Dm, n, q, pos)];
                for (int k = 0; k < q * n; ++k) {
                    ftab.push_back(Im[k]);
                    ftab.push_back(Dm[k]);
                }
            }
    ft.total = (int)ftab.size();
}

}  // namespace dg
