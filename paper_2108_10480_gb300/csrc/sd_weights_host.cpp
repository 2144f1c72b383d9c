// Triangle weight basis of App. C.3, solved on the host in double precision
// and converted to Bernstein-Bezier form for the kernels.
//
// The constraint system (10 point constraints and the normal-derivative
// equations on the three sides, App. C.3) is rank deficient; the paper takes
// the pseudoinverse solution. Here the minimum-norm solution is computed by
// modified Gram-Schmidt over the constraint rows: the orthonormal basis of the
// row space is built row by row, dependent rows are dropped, and the solution
// is the combination of the basis vectors that satisfies every kept row, so
// it lies in the row space and is therefore the minimum-norm solution.
//
// The kernels evaluate the weight in Bernstein form (degree 7 on the
// triangle, de Casteljau): its coefficients are of the size of the weight
// itself, whereas the monomial coefficients reach ~1e3 and lose ~1e-4 of
// relative accuracy in FP32.
#include <cmath>
#include <cstring>
#include <vector>

#include "sd.h"
#include "sd_wtab.h"

namespace sdw {

static const int NMON = 36;   // monomials phi1^a phi2^b, a + b <= 7

static void monomials(int (*ex)[2])
{
    int j = 0;
    for (int a = 0; a < 8; ++a)
        for (int b = 0; b < 8; ++b)
            if (a + b <= 7) { ex[j][0] = a; ex[j][1] = b; ++j; }
}

static double binom(int n, int k)
{
    if (k < 0 || k > n) return 0.0;
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

static double fact(int n)
{
    double r = 1.0;
    for (int i = 2; i <= n; ++i) r *= i;
    return r;
}

// Constraint rows (36 coefficients each) and right-hand sides for the three
// unit vectors of (1/v, 1/e, (v-1)/v).
static void constraint_system(std::vector<std::vector<double>>& rows, std::vector<std::vector<double>>& rhs)
{
    int ex[NMON][2];
    monomials(ex);
    auto point_row = [&](double x, double y, int col) {
        std::vector<double> r(NMON);
        for (int j = 0; j < NMON; ++j) r[j] = std::pow(x, ex[j][0]) * std::pow(y, ex[j][1]);
        std::vector<double> b(3, 0.0);
        b[col] = 1.0;
        rows.push_back(r); rhs.push_back(b);
    };
    const double t = 1.0 / 3.0;
    point_row(0, 0, 0); point_row(1, 0, 0); point_row(0, 1, 0);                 // vertices: 1/v
    point_row(t, 0, 1); point_row(2 * t, 0, 1); point_row(t, 2 * t, 1);          // two points per side: 1/e
    point_row(2 * t, t, 1); point_row(0, t, 1); point_row(0, 2 * t, 1);
    point_row(t, t, 2);                                                          // barycentre: (v-1)/v
    auto zero_rhs = std::vector<double>(3, 0.0);
    // d/dphi1 on phi1 = 0 is sum_b c_{1,b} phi2^b; d/dphi2 on phi2 = 0 likewise
    for (int j = 0; j < NMON; ++j) {
        if (ex[j][0] == 1) { std::vector<double> r(NMON, 0.0); r[j] = 1.0; rows.push_back(r); rhs.push_back(zero_rhs); }
        if (ex[j][1] == 1) { std::vector<double> r(NMON, 0.0); r[j] = 1.0; rows.push_back(r); rhs.push_back(zero_rhs); }
    }
    // (d/dphi1 + d/dphi2) on the hypotenuse, as a polynomial in t, for both
    // parametrisations (t, 1-t) and (1-t, t): each coefficient must vanish
    for (int swap = 0; swap < 2; ++swap) {
        std::vector<std::vector<double>> R(7, std::vector<double>(NMON, 0.0));
        for (int j = 0; j < NMON; ++j) {
            int a = ex[j][0], b = ex[j][1];
            const int terms[2][3] = {{a, a - 1, b}, {b, a, b - 1}};
            for (int s = 0; s < 2; ++s) {
                int coef = terms[s][0], p = terms[s][1], r = terms[s][2];
                if (coef == 0 || p < 0 || r < 0) continue;
                int tp = swap ? r : p, om = swap ? p : r;     // t^tp (1 - t)^om
                for (int k = 0; k <= om; ++k)
                    R[tp + k][j] += coef * binom(om, k) * ((k & 1) ? -1.0 : 1.0);
            }
        }
        for (int k = 0; k < 7; ++k) { rows.push_back(R[k]); rhs.push_back(zero_rhs); }
    }
}

// Minimum-norm solution of a consistent system by modified Gram-Schmidt
// with one re-orthogonalisation pass. x: [NMON][3].
static int min_norm_solve(const std::vector<std::vector<double>>& rows,
                          const std::vector<std::vector<double>>& rhs, double x[][3])
{
    std::vector<std::vector<double>> Q;
    std::vector<std::vector<double>> Y;
    for (size_t i = 0; i < rows.size(); ++i) {
        std::vector<double> u = rows[i];
        std::vector<double> c = rhs[i];
        double n0 = 0.0;
        for (double v : u) n0 += v * v;
        n0 = std::sqrt(n0);
        for (int pass = 0; pass < 2; ++pass)
            for (size_t k = 0; k < Q.size(); ++k) {
                double p = 0.0;
                for (int j = 0; j < NMON; ++j) p += u[j] * Q[k][j];
                for (int j = 0; j < NMON; ++j) u[j] -= p * Q[k][j];
                for (int m = 0; m < 3; ++m) c[m] -= p * Y[k][m];
            }
        double nr = 0.0;
        for (double v : u) nr += v * v;
        nr = std::sqrt(nr);
        if (nr > 1e-9 * n0) {
            for (double& v : u) v /= nr;
            for (double& v : c) v /= nr;
            Q.push_back(u);
            Y.push_back(c);
        }
    }
    for (int j = 0; j < NMON; ++j)
        for (int m = 0; m < 3; ++m) {
            double s = 0.0;
            for (size_t k = 0; k < Q.size(); ++k) s += Y[k][m] * Q[k][j];
            x[j][m] = s;
        }
    return (int)Q.size();
}

}  // namespace sdw

// Bernstein index of (i, j, k), i + j + k = 7: row r = j + k, then k.
static inline int bidx(int j, int k) { int r = j + k; return r * (r + 1) / 2 + k; }

extern "C" int sd_weight_basis(double* out)
{
    using namespace sdw;
    std::vector<std::vector<double>> rows, rhs;
    constraint_system(rows, rhs);
    double x[NMON][3];
    int rank = min_norm_solve(rows, rhs, x);
    if (rank != 30) return SD_ERR_INVALID_ARG;
    int ex[NMON][2];
    monomials(ex);
    std::memset(out, 0, sizeof(double) * 3 * 36);
    // phi1^a phi2^b = phi1^a phi2^b (phi0 + phi1 + phi2)^r, r = 7 - a - b,
    // expanded into B_ijk = 7!/(i! j! k!) phi0^i phi1^j phi2^k
    for (int m = 0; m < NMON; ++m) {
        int a = ex[m][0], b = ex[m][1], r = 7 - a - b;
        for (int j = a; j <= 7; ++j)
            for (int k = b; j + k <= 7; ++k) {
                int i = 7 - j - k;
                int jp = j - a, kp = k - b;
                if (i + jp + kp != r) continue;
                double mult = fact(r) / (fact(i) * fact(jp) * fact(kp));
                double conv = mult * fact(i) * fact(j) * fact(k) / fact(7);
                for (int c = 0; c < 3; ++c) out[c * 36 + bidx(j, k)] += x[m][c] * conv;
            }
    }
    return SD_OK;
}

// Nested-Horner tables of the blended triangle weight (App. C.3) for every
// class (v, e) with v = 1..SD_WT_VMAX, e = 1..SD_WT_EMAX: for each class and
// each orientation o (the barycentric taken as the base variable: phi_o),
// SD_WT_FLOATS floats:
//   36 coefficients of w~ = phi_o^7 sum_{a,b} c_ab x^a y^b,
//   28 of dw~/dphi1 and 28 of dw~/dphi2 (phi0 = 1 - phi1 - phi2, each
//      = phi_o^6 sum c_ab x^a y^b),
// where x, y are the ratios of the other two barycentrics (lower index
// first) to phi_o, c_ab = (Bernstein coefficient) x (multinomial), and the
// coefficients run in Horner order: powers of y from high to low outer,
// powers of x from high to low inner. Computed in FP64 from the basis of
// sd_weight_basis, rounded to fp32 once.
// the Horner tables (3 orientations x SD_WT_FLOATS floats) of one weight
// polynomial with Bernstein coefficients w(n) = a_v basis_V + a_e basis_E +
// a_b basis_B
static float* horner_tables(const double* basis, double a_v, double a_e, double a_b, float* o_ptr)
{
    auto fact = [](int n) { double f = 1.0; for (int i = 2; i <= n; ++i) f *= i; return f; };
    auto multi = [&](int n, int i, int j, int k) { return fact(n) / (fact(i) * fact(j) * fact(k)); };
    {
        {
            // degree-7 coefficients b[i][j][k] and the degree-6 differences
            double b7[8][8][8] = {}, d1[7][7][7] = {}, d2[7][7][7] = {};
            for (int j = 0; j <= 7; ++j)
                for (int k = 0; j + k <= 7; ++k) {
                    const int n = bidx(j, k), i = 7 - j - k;
                    b7[i][j][k] = a_v * basis[n] + a_e * basis[36 + n] + a_b * basis[72 + n];
                }
            for (int j = 0; j <= 6; ++j)
                for (int k = 0; j + k <= 6; ++k) {
                    const int i = 6 - j - k;
                    d1[i][j][k] = 7.0 * (b7[i][j + 1][k] - b7[i + 1][j][k]);
                    d2[i][j][k] = 7.0 * (b7[i][j][k + 1] - b7[i + 1][j][k]);
                }
            for (int o = 0; o < 3; ++o) {
                const int x0 = o == 0 ? 1 : 0, y0 = o == 2 ? 1 : 2;    // the other two variables
                auto emit = [&](int deg, auto coef) {
                    for (int bp = deg; bp >= 0; --bp)
                        for (int ap = deg - bp; ap >= 0; --ap) {
                            int ex[3];
                            ex[o] = deg - ap - bp;
                            ex[x0] = ap;
                            ex[y0] = bp;
                            *o_ptr++ = (float)(coef(ex[0], ex[1], ex[2]) * multi(deg, ex[0], ex[1], ex[2]));
                        }
                };
                emit(7, [&](int i, int j, int k) { return b7[i][j][k]; });
                emit(6, [&](int i, int j, int k) { return d1[i][j][k]; });
                emit(6, [&](int i, int j, int k) { return d2[i][j][k]; });
            }
        }
    }
    return o_ptr;
}

extern "C" int sd_weight_horner_tables(float* out)
{
    double basis[108];
    int rc = sd_weight_basis(basis);
    if (rc != SD_OK) return rc;
    float* o_ptr = out;
    for (int v = 1; v <= SD_WT_VMAX; ++v)
        for (int e = 1; e <= SD_WT_EMAX; ++e)
            o_ptr = horner_tables(basis, 1.0 / v, 1.0 / e, (v - 1.0) / v, o_ptr);
    return (int)(o_ptr - out) == SD_WT_VMAX * SD_WT_EMAX * 3 * SD_WT_FLOATS ? SD_OK : SD_ERR_INVALID_ARG;
}

int sd_weight_horner_basis(float* out)
{
    double basis[108];
    int rc = sd_weight_basis(basis);
    if (rc != SD_OK) return rc;
    // w~ = base + (1/v) dv + (1/e) de with base = P_B, dv = P_V - P_B, de = P_E
    float* o_ptr = horner_tables(basis, 0.0, 0.0, 1.0, out);
    o_ptr = horner_tables(basis, 1.0, 0.0, -1.0, o_ptr);
    o_ptr = horner_tables(basis, 0.0, 1.0, 0.0, o_ptr);
    return (int)(o_ptr - out) == 3 * 3 * SD_WT_FLOATS ? SD_OK : SD_ERR_INVALID_ARG;
}
