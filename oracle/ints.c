/*
 * Oracle (test infrastructure only): plain FP64 integrals over contracted
 * Cartesian Gaussian shells.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load this file's library; the product path
 * never does.
 *
 * The paper's iteration 0 precomputes V, T, S and the two-electron tensor
 * I^2e (Section 3.1, Eq. 1).  Here those integrals are evaluated by the
 * McMurchie-Davidson Hermite-Gaussian scheme (textbook form: Hermite
 * expansion coefficients E_t^{ij}, Hermite Coulomb integrals R_{tuv}^n and the
 * Boys function F_n), which is deliberately a different route from the
 * Obara-Saika/Head-Gordon-Pople recursion of the CUDA kernels.
 *
 * Shells are passed as flat arrays: centre xyz (bohr), angular momentum l,
 * number of primitives, exponents and contraction coefficients (the
 * coefficients already carry primitive normalisation and the contracted
 * renormalisation; see oracle/basis.py).  Cartesian components of a shell
 * with angular momentum l are ordered lx descending, then ly descending
 * (for l = 1: x, y, z).  Every routine here is O(plain): no screening at the
 * primitive level, no reuse beyond what the recursions define.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define LMAXE 4   /* max l per index in E tables (kinetic needs l_b + 2) */
#define LTOT 8    /* max total Hermite order in R tables */
#define MAXP 8    /* max primitives per shell */

/* ---------------------------------------------------------------- Boys */
/* F_m(T) = int_0^1 t^(2m) exp(-T t^2) dt.
 * T < 30: convergent series F_m(T) = exp(-T) sum_k (2T)^k / prod_{i=0..k}(2m+2i+1)
 * (all terms positive).  T >= 30: F_0 = (1/2) sqrt(pi/T) erf(sqrt(T)) and
 * the upward recursion F_{m+1} = ((2m+1) F_m - exp(-T)) / (2T), which is stable
 * there because exp(-T) is negligible against (2m+1) F_m. */
double oracle_boys(int m, double T)
{
    if (T < 1e-300)
        return 1.0 / (2 * m + 1);
    if (T < 30.0) {
        double term = 1.0 / (2 * m + 1);
        double sum = term;
        for (int k = 1; k < 400; k++) {
            term *= 2.0 * T / (2 * m + 2 * k + 1);
            sum += term;
            if (term < 1e-18 * sum)
                break;
        }
        return exp(-T) * sum;
    }
    double f = 0.5 * sqrt(M_PI / T) * erf(sqrt(T));
    double e = exp(-T);
    for (int k = 0; k < m; k++)
        f = ((2 * k + 1) * f - e) / (2.0 * T);
    return f;
}

/* ------------------------------------------------- Hermite coefficients */
/* E_t^{ij} for one Cartesian direction; Qx = A_x - B_x.  Textbook recursion
 * in i (j = 0) and then in j:
 *   E_t^{i+1,j} = E_{t-1}^{ij}/(2p) + X_PA E_t^{ij} + (t+1) E_{t+1}^{ij}
 *   E_t^{i,j+1} = E_{t-1}^{ij}/(2p) + X_PB E_t^{ij} + (t+1) E_{t+1}^{ij}
 * with X_PA = -(b/p) Qx, X_PB = (a/p) Qx and E_0^{00} = exp(-ab/p Qx^2). */
static double herm_E(int i, int j, int t, double Qx, double a, double b)
{
    double p = a + b;
    if (t < 0 || t > i + j || i < 0 || j < 0)
        return 0.0;
    if (i == 0 && j == 0)
        return exp(-a * b / p * Qx * Qx);
    if (j == 0)
        return herm_E(i - 1, j, t - 1, Qx, a, b) / (2 * p)
               - (b / p) * Qx * herm_E(i - 1, j, t, Qx, a, b)
               + (t + 1) * herm_E(i - 1, j, t + 1, Qx, a, b);
    return herm_E(i, j - 1, t - 1, Qx, a, b) / (2 * p)
           + (a / p) * Qx * herm_E(i, j - 1, t, Qx, a, b)
           + (t + 1) * herm_E(i, j - 1, t + 1, Qx, a, b);
}

/* ------------------------------------------- Hermite Coulomb integrals */
/* R_{tuv}^n(alpha, X, Y, Z):  R_{000}^n = (-2 alpha)^n F_n(alpha R^2),
 *   R_{t+1,u,v}^n = t R_{t-1,u,v}^{n+1} + X R_{tuv}^{n+1}  (same in u, v).
 * Filled for all t+u+v+n <= L; table index [n][t][u][v]. */
typedef struct {
    double v[LTOT + 1][LTOT + 1][LTOT + 1][LTOT + 1];
} rtab_t;

static void fill_R(rtab_t *R, int L, double alpha, double X, double Y, double Z)
{
    double T = alpha * (X * X + Y * Y + Z * Z);
    for (int n = L; n >= 0; n--) {
        double fac = 1.0;
        for (int k = 0; k < n; k++)
            fac *= -2.0 * alpha;
        R->v[n][0][0][0] = fac * oracle_boys(n, T);
        for (int s = 1; s <= L - n; s++)
            for (int t = 0; t <= s; t++)
                for (int u = 0; u <= s - t; u++) {
                    int w = s - t - u;
                    double r;
                    if (t > 0)
                        r = (t > 1 ? (t - 1) * R->v[n + 1][t - 2][u][w] : 0.0)
                            + X * R->v[n + 1][t - 1][u][w];
                    else if (u > 0)
                        r = (u > 1 ? (u - 1) * R->v[n + 1][t][u - 2][w] : 0.0)
                            + Y * R->v[n + 1][t][u - 1][w];
                    else
                        r = (w > 1 ? (w - 1) * R->v[n + 1][t][u][w - 2] : 0.0)
                            + Z * R->v[n + 1][t][u][w - 1];
                    R->v[n][t][u][w] = r;
                }
    }
}

/* ------------------------------------------------------------- shells */
static int ncart(int l) { return (l + 1) * (l + 2) / 2; }

static void cart(int l, int c, int *lx, int *ly, int *lz)
{
    int k = 0;
    *lx = *ly = *lz = 0;
    for (int x = l; x >= 0; x--)
        for (int y = l - x; y >= 0; y--) {
            if (k == c) {
                *lx = x;
                *ly = y;
                *lz = l - x - y;
                return;
            }
            k++;
        }
}

/* ---------------------------------------------------- one-electron ints */
/* Primitive overlap in one direction: S_ij = E_0^{ij} sqrt(pi/p). */
static double s1d(int i, int j, double Qx, double a, double b)
{
    if (i < 0 || j < 0)
        return 0.0;
    return herm_E(i, j, 0, Qx, a, b) * sqrt(M_PI / (a + b));
}

/* Primitive kinetic in one direction (acting on the ket):
 * T_ij = -2 b^2 S_{i,j+2} + b (2j+1) S_ij - (1/2) j (j-1) S_{i,j-2}. */
static double t1d(int i, int j, double Qx, double a, double b)
{
    return -2.0 * b * b * s1d(i, j + 2, Qx, a, b) + b * (2 * j + 1) * s1d(i, j, Qx, a, b)
           - 0.5 * j * (j - 1) * s1d(i, j - 2, Qx, a, b);
}

/* S, T and V (nuclear attraction, sum over point charges Zc at Cxyz) for the
 * whole basis; ao0[s] is the first AO index of shell s, nbf the AO count.
 * Outputs are nbf x nbf row-major. */
void oracle_one_electron(int nsh, const double *xyz, const int *l, const int *np,
                         const double *ex, const double *co, const int *ao0, int nbf,
                         int ncharge, const double *Zc, const double *Cxyz,
                         double *S, double *T, double *V)
{
    memset(S, 0, sizeof(double) * nbf * nbf);
    memset(T, 0, sizeof(double) * nbf * nbf);
    memset(V, 0, sizeof(double) * nbf * nbf);
    for (int P = 0; P < nsh; P++)
        for (int Q = 0; Q < nsh; Q++) {
            const double *A = xyz + 3 * P, *B = xyz + 3 * Q;
            for (int ca = 0; ca < ncart(l[P]); ca++)
                for (int cb = 0; cb < ncart(l[Q]); cb++) {
                    int ax, ay, az, bx, by, bz;
                    cart(l[P], ca, &ax, &ay, &az);
                    cart(l[Q], cb, &bx, &by, &bz);
                    double s = 0, t = 0, v = 0;
                    for (int pa = 0; pa < np[P]; pa++)
                        for (int pb = 0; pb < np[Q]; pb++) {
                            double a = ex[P * MAXP + pa], b = ex[Q * MAXP + pb];
                            double cc = co[P * MAXP + pa] * co[Q * MAXP + pb];
                            double p = a + b;
                            double sx = s1d(ax, bx, A[0] - B[0], a, b);
                            double sy = s1d(ay, by, A[1] - B[1], a, b);
                            double sz = s1d(az, bz, A[2] - B[2], a, b);
                            s += cc * sx * sy * sz;
                            t += cc * (t1d(ax, bx, A[0] - B[0], a, b) * sy * sz
                                       + sx * t1d(ay, by, A[1] - B[1], a, b) * sz
                                       + sx * sy * t1d(az, bz, A[2] - B[2], a, b));
                            double Px = (a * A[0] + b * B[0]) / p;
                            double Py = (a * A[1] + b * B[1]) / p;
                            double Pz = (a * A[2] + b * B[2]) / p;
                            for (int c = 0; c < ncharge; c++) {
                                rtab_t R;
                                int L = l[P] + l[Q];
                                fill_R(&R, L, p, Px - Cxyz[3 * c], Py - Cxyz[3 * c + 1],
                                       Pz - Cxyz[3 * c + 2]);
                                double acc = 0;
                                for (int tt = 0; tt <= ax + bx; tt++)
                                    for (int uu = 0; uu <= ay + by; uu++)
                                        for (int ww = 0; ww <= az + bz; ww++)
                                            acc += herm_E(ax, bx, tt, A[0] - B[0], a, b)
                                                   * herm_E(ay, by, uu, A[1] - B[1], a, b)
                                                   * herm_E(az, bz, ww, A[2] - B[2], a, b)
                                                   * R.v[0][tt][uu][ww];
                                v += -Zc[c] * cc * (2.0 * M_PI / p) * acc;
                            }
                        }
                    int i = ao0[P] + ca, j = ao0[Q] + cb;
                    S[i * nbf + j] = s;
                    T[i * nbf + j] = t;
                    V[i * nbf + j] = v;
                }
        }
}

/* -------------------------------------------------------------- ERIs */
/* One contracted shell-quartet block (PQ|RS) in chemists' notation,
 * (ab|cd) = int a(1) b(1) r12^-1 c(2) d(2).  Primitive formula:
 *   2 pi^(5/2) / (p q sqrt(p+q)) sum_{tuv} E^{ab}_{tuv} sum_{t'u'v'}
 *   (-1)^{t'+u'+v'} E^{cd}_{t'u'v'} R_{t+t',u+u',v+v'}(p q/(p+q), P - Q).
 * out is row-major [na][nb][nc][nd]. */
void oracle_eri_block(int P, int Q, int Rs, int Ss, const double *xyz, const int *l,
                      const int *np, const double *ex, const double *co, double *out)
{
    int sh[4] = {P, Q, Rs, Ss};
    int n[4];
    for (int k = 0; k < 4; k++)
        n[k] = ncart(l[sh[k]]);
    int ntot = n[0] * n[1] * n[2] * n[3];
    for (int k = 0; k < ntot; k++)
        out[k] = 0.0;
    const double *A = xyz + 3 * P, *B = xyz + 3 * Q, *C = xyz + 3 * Rs, *D = xyz + 3 * Ss;
    int L = l[P] + l[Q] + l[Rs] + l[Ss];
    /* Hermite coefficients of the bra and ket primitive pairs, tabulated once
     * per pair: E[dir][i][j][t]. */
    double Eab[3][LMAXE + 1][LMAXE + 1][2 * LMAXE + 1];
    double Ecd[3][LMAXE + 1][LMAXE + 1][2 * LMAXE + 1];
    for (int pa = 0; pa < np[P]; pa++)
        for (int pb = 0; pb < np[Q]; pb++) {
            double a = ex[P * MAXP + pa], b = ex[Q * MAXP + pb];
            for (int k = 0; k < 3; k++)
                for (int i = 0; i <= l[P]; i++)
                    for (int j = 0; j <= l[Q]; j++)
                        for (int t = 0; t <= i + j; t++)
                            Eab[k][i][j][t] = herm_E(i, j, t, A[k] - B[k], a, b);
            for (int pc = 0; pc < np[Rs]; pc++)
                for (int pd = 0; pd < np[Ss]; pd++) {
                    double c = ex[Rs * MAXP + pc], d = ex[Ss * MAXP + pd];
                    for (int k = 0; k < 3; k++)
                        for (int i = 0; i <= l[Rs]; i++)
                            for (int j = 0; j <= l[Ss]; j++)
                                for (int t = 0; t <= i + j; t++)
                                    Ecd[k][i][j][t] = herm_E(i, j, t, C[k] - D[k], c, d);
                    double cc = co[P * MAXP + pa] * co[Q * MAXP + pb] * co[Rs * MAXP + pc]
                                * co[Ss * MAXP + pd];
                    double p = a + b, q = c + d, alpha = p * q / (p + q);
                    double Pc[3], Qc[3];
                    for (int k = 0; k < 3; k++) {
                        Pc[k] = (a * A[k] + b * B[k]) / p;
                        Qc[k] = (c * C[k] + d * D[k]) / q;
                    }
                    rtab_t R;
                    fill_R(&R, L, alpha, Pc[0] - Qc[0], Pc[1] - Qc[1], Pc[2] - Qc[2]);
                    double pref = 2.0 * pow(M_PI, 2.5) / (p * q * sqrt(p + q)) * cc;
                    int idx = 0;
                    for (int ia = 0; ia < n[0]; ia++)
                        for (int ib = 0; ib < n[1]; ib++)
                            for (int ic = 0; ic < n[2]; ic++)
                                for (int id = 0; id < n[3]; id++, idx++) {
                                    int a3[3], b3[3], c3[3], d3[3];
                                    cart(l[P], ia, &a3[0], &a3[1], &a3[2]);
                                    cart(l[Q], ib, &b3[0], &b3[1], &b3[2]);
                                    cart(l[Rs], ic, &c3[0], &c3[1], &c3[2]);
                                    cart(l[Ss], id, &d3[0], &d3[1], &d3[2]);
                                    double acc = 0;
                                    for (int t = 0; t <= a3[0] + b3[0]; t++)
                                        for (int u = 0; u <= a3[1] + b3[1]; u++)
                                            for (int v = 0; v <= a3[2] + b3[2]; v++) {
                                                double eab = Eab[0][a3[0]][b3[0]][t]
                                                             * Eab[1][a3[1]][b3[1]][u]
                                                             * Eab[2][a3[2]][b3[2]][v];
                                                for (int t2 = 0; t2 <= c3[0] + d3[0]; t2++)
                                                    for (int u2 = 0; u2 <= c3[1] + d3[1]; u2++)
                                                        for (int v2 = 0; v2 <= c3[2] + d3[2]; v2++) {
                                                            double ecd = Ecd[0][c3[0]][d3[0]][t2]
                                                                         * Ecd[1][c3[1]][d3[1]][u2]
                                                                         * Ecd[2][c3[2]][d3[2]][v2];
                                                            double sgn = ((t2 + u2 + v2) & 1) ? -1.0 : 1.0;
                                                            acc += eab * sgn * ecd * R.v[0][t + t2][u + u2][v + v2];
                                                        }
                                            }
                                    out[idx] += pref * acc;
                                }
                }
        }
}

/* Blocks for a list of shell quartets (4 ints each), written at the given
 * element offsets of out. */
void oracle_eri_blocks(int nq, const int *quart, const int64_t *off, const double *xyz,
                       const int *l, const int *np, const double *ex, const double *co,
                       double *out)
{
    for (int k = 0; k < nq; k++)
        oracle_eri_block(quart[4 * k], quart[4 * k + 1], quart[4 * k + 2], quart[4 * k + 3],
                         xyz, l, np, ex, co, out + off[k]);
}
