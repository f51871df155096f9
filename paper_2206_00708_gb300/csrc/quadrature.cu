// Quadrature tables of the library (paper Sec. 5.1: rules of order four with the
// Sauter-Schwab transformations for singular pairs).
//
// * Regular pairs: the fully symmetric 6-point triangle rule exact to degree 4
//   (two orbits of barycentric points (a, a, 1-2a)).  Starting from the values
//   published by Dunavant (1985), the four parameters are refined here by Newton's
//   method on the exact moments of the invariant polynomials 1, e2, e3, e2^2, so
//   the table is exact to double rounding.
// * Singular pairs: Gauss-Legendre nodes on [0,1] by Newton iteration on the
//   Legendre three-term recurrence, and the Sauter-Schwab regularising maps of
//   [0,1]^4 onto T^ x T^ (T^ = {0 <= x2 <= x1 <= 1}): coincident pairs 6 regions,
//   edge-adjacent pairs 4 regions (the half x1 >= y1 split by the plane
//   x2 = x1 - y1 + y2, and its mirror), vertex-adjacent pairs 2 regions.
#include "bem_internal.cuh"

#include <cmath>
#include <map>
#include <memory>
#include <mutex>

namespace bem {

namespace {

// exact integrals over the reference triangle of the S3-invariant polynomials
// 1, e2 = l0 l1 + l1 l2 + l2 l0, e3 = l0 l1 l2, e2^2 (barycentric l).
void moments_of(double a, double out[4]) {
    double b = 1.0 - 2.0 * a;
    double e2 = a * a + 2.0 * a * b;
    double e3 = a * a * b;
    out[0] = 1.0;
    out[1] = e2;
    out[2] = e3;
    out[3] = e2 * e2;
}

TriRule build_rule() {
    // exact moments: int l0^i l1^j l2^k = 2 i! j! k! / (i+j+k+2)! times area 1/2
    // int 1 = 1/2; int e2 = 3 * 1/24 = 1/8; int e3 = 1/120; int e2^2:
    //   e2^2 = sum over 3 terms (li lj)^2 + 2 * sum over 3 cross terms li^2 lj lk
    //   int (l0 l1)^2 = 2*2*2/720 * 1/2 ... computed from the factorial formula below.
    auto mono = [](int i, int j, int k) {
        double f[9] = {1, 1, 2, 6, 24, 120, 720, 5040, 40320};
        return f[i] * f[j] * f[k] / f[i + j + k + 2];  // over the triangle of area 1/2
    };
    double target[4];
    target[0] = mono(0, 0, 0);
    target[1] = 3.0 * mono(1, 1, 0);
    target[2] = mono(1, 1, 1);
    target[3] = 3.0 * mono(2, 2, 0) + 6.0 * mono(2, 1, 1);
    // Dunavant's degree-4 values (weights normalised to total 1)
    double p[4] = {0.445948490915965, 0.223381589678011 * 0.5, 0.091576213509771,
                   0.109951743655322 * 0.5};
    for (int it = 0; it < 50; ++it) {
        double r[4], m1[4], m2[4];
        moments_of(p[0], m1);
        moments_of(p[2], m2);
        for (int i = 0; i < 4; ++i) r[i] = 3.0 * (p[1] * m1[i] + p[3] * m2[i]) - target[i];
        double Jm[4][4];
        for (int c = 0; c < 4; ++c) {
            double h = (c % 2 == 0) ? 1e-7 : 1e-8;
            double q[4] = {p[0], p[1], p[2], p[3]};
            q[c] += h;
            double a1[4], a2[4];
            moments_of(q[0], a1);
            moments_of(q[2], a2);
            double rp[4];
            for (int i = 0; i < 4; ++i) rp[i] = 3.0 * (q[1] * a1[i] + q[3] * a2[i]) - target[i];
            q[c] -= 2 * h;
            moments_of(q[0], a1);
            moments_of(q[2], a2);
            for (int i = 0; i < 4; ++i) {
                double rm = 3.0 * (q[1] * a1[i] + q[3] * a2[i]) - target[i];
                Jm[i][c] = (rp[i] - rm) / (2 * h);
            }
        }
        // solve Jm dx = -r by Gaussian elimination with partial pivoting
        double A[4][5];
        for (int i = 0; i < 4; ++i) {
            for (int c = 0; c < 4; ++c) A[i][c] = Jm[i][c];
            A[i][4] = -r[i];
        }
        for (int c = 0; c < 4; ++c) {
            int piv = c;
            for (int i = c + 1; i < 4; ++i)
                if (std::fabs(A[i][c]) > std::fabs(A[piv][c])) piv = i;
            for (int k = 0; k < 5; ++k) std::swap(A[c][k], A[piv][k]);
            for (int i = c + 1; i < 4; ++i) {
                double f = A[i][c] / A[c][c];
                for (int k = c; k < 5; ++k) A[i][k] -= f * A[c][k];
            }
        }
        double dx[4];
        for (int i = 3; i >= 0; --i) {
            double s = A[i][4];
            for (int k = i + 1; k < 4; ++k) s -= A[i][k] * dx[k];
            dx[i] = s / A[i][i];
        }
        double mx = 0;
        for (int i = 0; i < 4; ++i) {
            p[i] += dx[i];
            mx = std::fmax(mx, std::fabs(dx[i]));
        }
        if (mx < 1e-17) break;
    }
    TriRule R;
    const double a[2] = {p[0], p[2]}, w[2] = {p[1], p[3]};
    for (int o = 0; o < 2; ++o) {
        double b = 1.0 - 2.0 * a[o];
        // barycentric (l0, l1, l2) = (a, a, b), (a, b, a), (b, a, a); (s, t) = (l1, l2)
        double l1[3] = {a[o], b, a[o]}, l2[3] = {b, a[o], a[o]};
        for (int m = 0; m < 3; ++m) {
            R.s[3 * o + m] = l1[m];
            R.t[3 * o + m] = l2[m];
            R.w[3 * o + m] = w[o];
        }
    }
    return R;
}

// Gauss-Legendre on [0,1]: Newton on P_n with the three-term recurrence.
void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w) {
    x.resize(n);
    w.resize(n);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < n; ++i) {
        double z = std::cos(pi * (i + 0.75) / (n + 0.5));
        double dp = 0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = pk;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        // recompute derivative at the converged node
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = pk;
        }
        if (n == 1) { p1 = z; p0 = 1.0; }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = 0.5 * (1.0 - z);
        w[i] = 1.0 / ((1.0 - z * z) * dp * dp);  // = 0.5 * 2/((1-z^2) P'^2)
    }
}

void push(std::vector<double>& t, double x1, double x2, double y1, double y2, double w) {
    t.push_back(x1); t.push_back(x2); t.push_back(y1); t.push_back(y2); t.push_back(w);
}

void build_ss(int n, SSTable& T) {
    std::vector<double> g, gw;
    gauss_legendre01(n, g, gw);
    T.n = n;
    T.host.clear();
    // coincident: Jacobian xi^3 e1^2 e2, six regions
    for (int a = 0; a < n; ++a) for (int b = 0; b < n; ++b) for (int c = 0; c < n; ++c) for (int d = 0; d < n; ++d) {
        double xi = g[a], e1 = g[b], e2 = g[c], e3 = g[d];
        double w = gw[a] * gw[b] * gw[c] * gw[d] * xi * xi * xi * e1 * e1 * e2;
        double A1 = xi, A2 = xi * (1 - e1 + e1 * e2), B1 = xi * (1 - e1 * e2 * e3), B2 = xi * (1 - e1);
        push(T.host, A1, A2, B1, B2, w);
        push(T.host, B1, B2, A1, A2, w);
        double C1 = xi, C2 = xi * e1 * (1 - e2 + e2 * e3), D1 = xi * (1 - e1 * e2), D2 = xi * e1 * (1 - e2);
        push(T.host, C1, C2, D1, D2, w);
        push(T.host, D1, D2, C1, C2, w);
        double E1 = xi * (1 - e1 * e2 * e3), E2 = xi * e1 * (1 - e2 * e3), F1 = xi, F2 = xi * e1 * (1 - e2);
        push(T.host, E1, E2, F1, F2, w);
        push(T.host, F1, F2, E1, E2, w);
    }
    T.count[0] = (int)(T.host.size() / 5);
    // edge-adjacent: common edge x2 = 0 = y2 with x1 = y1 on it; four regions
    for (int a = 0; a < n; ++a) for (int b = 0; b < n; ++b) for (int c = 0; c < n; ++c) for (int d = 0; d < n; ++d) {
        double xi = g[a], e1 = g[b], e2 = g[c], e3 = g[d];
        double w1 = gw[a] * gw[b] * gw[c] * gw[d] * xi * xi * xi * e1 * e1;
        double w2 = w1 * e2;
        // region x1 >= y1, x2 <= x1 - y1 + y2
        double P1 = xi, P2 = xi * e1 * e3, Q1 = xi * (1 - e1 * e2), Q2 = xi * e1 * (1 - e2);
        // region x1 >= y1, x2 >= x1 - y1 + y2
        double R1 = xi, R2 = xi * e1, S1 = xi * (1 - e1 * e2 * e3), S2 = xi * e1 * e2 * (1 - e3);
        push(T.host, P1, P2, Q1, Q2, w1);
        push(T.host, R1, R2, S1, S2, w2);
        push(T.host, Q1, Q2, P1, P2, w1);
        push(T.host, S1, S2, R1, R2, w2);
    }
    T.count[1] = (int)(T.host.size() / 5) - T.count[0];
    // vertex-adjacent: common vertex at x^ = 0 = y^; two regions, Jacobian xi^3 e2
    for (int a = 0; a < n; ++a) for (int b = 0; b < n; ++b) for (int c = 0; c < n; ++c) for (int d = 0; d < n; ++d) {
        double xi = g[a], e1 = g[b], e2 = g[c], e3 = g[d];
        double w = gw[a] * gw[b] * gw[c] * gw[d] * xi * xi * xi * e2;
        push(T.host, xi, xi * e1, xi * e2, xi * e2 * e3, w);
        push(T.host, xi * e2, xi * e2 * e1, xi, xi * e3, w);
    }
    T.count[2] = (int)(T.host.size() / 5) - T.count[0] - T.count[1];
    T.offset[0] = 0;
    T.offset[1] = T.count[0];
    T.offset[2] = T.count[0] + T.count[1];
}

std::mutex g_ss_mutex;
std::map<std::pair<int, int>, std::unique_ptr<SSTable>> g_ss;  // (device, n)

}  // namespace

const TriRule& tri_rule_degree4() {
    static const TriRule R = build_rule();
    return R;
}

bem_status ss_table_get(int n, cudaStream_t stream, const double** dev_ptr, int count[3], int offset[3]) {
    int dev = 0;
    BEM_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_ss_mutex);
    auto key = std::make_pair(dev, n);
    auto it = g_ss.find(key);
    if (it == g_ss.end()) {
        auto T = std::make_unique<SSTable>();
        build_ss(n, *T);
        size_t bytes = T->host.size() * sizeof(double);
        // tables live for the life of the process: allocate outside any stream order
        BEM_CUDA_TRY(cudaMalloc(&T->dev.p, bytes));
        T->dev.bytes = bytes;
        T->dev.stream = nullptr;
        BEM_CUDA_TRY(cudaMemcpy(T->dev.p, T->host.data(), bytes, cudaMemcpyHostToDevice));
        it = g_ss.emplace(key, std::move(T)).first;
    }
    *dev_ptr = it->second->dev.as<double>();
    for (int i = 0; i < 3; ++i) {
        count[i] = it->second->count[i];
        offset[i] = it->second->offset[i];
    }
    (void)stream;
    return BEM_OK;
}

}  // namespace bem
