/*
 * lbm_oracle.c -- plain FP64 CPU oracle for the second-order force scheme of
 * Li, Duan & Shan, "Second-order force scheme for lattice Boltzmann method"
 * (arXiv:2212.07494).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * statement of what the GPU path computes.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, table or header with the CUDA path.
 *
 * Everything is written the way the paper states it: full Hermite tensors
 * (all D^n components, not only the independent ones), moments obtained by
 * the discrete transform of Eq. (dft), frame shifts written as sums over the
 * distinct index placements of the symmetric products (Sec. II.C, Eq. bbd1),
 * collide then push-stream (Sec. II.C, last equation).  Hermite units are used
 * inside (xi_i = sqrt(3) c_i, u_H = sqrt(3) u, g_H = sqrt(3) g, theta = 1,
 * dt = 1); the interface takes lattice units.
 *
 * Readings of the paper taken here (each documented in the design notes):
 *  - tau values are the tau-hat of Eq. (explict_eq): tau_hat = tau + 1/2.
 *  - SMRT uses one relaxation time per Hermite order (tau_nk = tau_n).
 *  - the force keeps only its equilibrium part in the co-moving frame:
 *    d_F^(1) = rho g, d_F^(n>=2) = 0 (Sec. II.C, after Eq. Frc).  The third
 *    collision mode (OR_SMRT_FNEQ) keeps the non-equilibrium parts as well,
 *    d_F^(n) = n g d^(n-1) for n <= 4 (Eq. Frc, third and fourth terms), with
 *    d^(n-1) the moments of f itself, recovered from those of fbar by
 *    inverting Eq. (newf) order by order.
 *  - the second-order relaxation of both SMRT forms may split into the
 *    traceless (shear) part and the trace (bulk) part, tau_{2,2} = tau[2] and
 *    tau_{2,0} = tau_bulk (Eq. domg).  Orders 3 and 4 keep one tau each: their
 *    trace parts need components the lattices do not carry.
 *  - the fourth collision mode (OR_MRT_RAW) is the raw-moment MRT of the
 *    appendix: per-order relaxation of the raw non-equilibrium moments, the
 *    fourth order from the appendix's recursion, the force's equilibrium part
 *    a_F^(n) = n F u^(n-1) only.
 *  - retained Hermite components per lattice: D2Q9/D3Q27 keep components with
 *    per-axis multiplicity <= 2 and order <= 4; D3Q19 keeps orders <= 2 and
 *    the six (2,1,0) third-order components.  D3Q19 is a degree-5 rule, so a
 *    fourth-order component times a second-order one is not integrated
 *    exactly: the (2,2,0) components would leak into the stress and are not
 *    kept.  Components outside the set are dropped from equilibrium and
 *    non-equilibrium parts alike.
 *  - BGK uses the second-order equilibrium and force of Eq. (collision_BGK)
 *    and the second-order F(xi) (Sec. II.A).
 *  - initial state: fbar = f_eq(rho0,u0) - F/2 (zero non-equilibrium part).
 *  - the state is stored as deviations delta_i = fbar_i - w_i (see the
 *    collision section).
 *  - boundaries: periodic, or halfway bounce-back at -1/2 and n-1/2 and at
 *    solid nodes.
 *
 * Pins: every computation here is checked by CPU tests (tests/test_oracle_*)
 * against something other than itself -- quadrature and orthogonality
 * identities, exact transform and shift identities, the textbook Guo update,
 * the trapezoidal rule restated in population space (D2Q9, D3Q27), raw-moment
 * relaxation at one relaxation time (D3Q19), brute-force streaming, and
 * closed-form flows (Poiseuille with its wall slip, Kolmogorov, shear and
 * sound waves, Taylor-Green, Womersley).  No function is parity unpinned.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXQ 27
#define OR_MAXN 4
/* offsets of order-n tensors inside a packed moment vector: 1 + D + D^2 + ... */
#define OR_PACK 121 /* 1 + 3 + 9 + 27 + 81 for D = 3 */

enum { OR_D2Q9 = 0, OR_D3Q19 = 1, OR_D3Q27 = 2 };
enum { OR_BGK = 0, OR_SMRT = 1, OR_SMRT_FNEQ = 2, OR_MRT_RAW = 3 };

typedef struct {
    int id, D, Q;
    int c[OR_MAXQ][3];
    double w[OR_MAXQ];
    double xi[OR_MAXQ][3];       /* Hermite-unit abscissas, sqrt(3) c_i */
    int opp[OR_MAXQ];
    int off[OR_MAXN + 2];        /* packed tensor offsets, off[n] .. off[n+1] */
    double H[OR_MAXQ][OR_PACK];  /* H^(n)(xi_i), all components, packed */
    unsigned char keep[OR_PACK]; /* retained-component mask, packed */
    int order[OR_PACK];          /* order n of each packed component */
    int dig[OR_PACK][4];         /* its index tuple (a1..an) */
    int rest[OR_PACK][16];       /* packed index of the tuple with the positions of
                                    subset S removed (see shift) */
} or_lattice;

static const double SQ3 = 1.7320508075688772935274463415059;

/* ------------------------------------------------------------------------ */
/* Lattices.  The paper names no weights or abscissas; these are the usual   */
/* Gauss-Hermite rules (D1Q3 = {0, +-sqrt3} with weights {2/3, 1/6, 1/6}).   */
/* Population order (shared convention of the whole library):                 */
/*  D2Q9 : 0 rest; 1..4 (1,0) (0,1) (-1,0) (0,-1); 5..8 (1,1) (-1,1) (-1,-1)  */
/*         (1,-1)                                                             */
/*  D3Q19: 0 rest; 1..6 faces +-x, +-y, +-z; 7..18 edges in opposite pairs    */
/*  D3Q27: D3Q19 then 8 corners in opposite pairs                             */
/* ------------------------------------------------------------------------ */
static const int C2Q9[9][3] = {{0,0,0},{1,0,0},{0,1,0},{-1,0,0},{0,-1,0},
                               {1,1,0},{-1,1,0},{-1,-1,0},{1,-1,0}};
static const int C3Q27[27][3] = {
    {0,0,0},
    {1,0,0},{-1,0,0},{0,1,0},{0,-1,0},{0,0,1},{0,0,-1},
    {1,1,0},{-1,-1,0},{1,-1,0},{-1,1,0},
    {1,0,1},{-1,0,-1},{1,0,-1},{-1,0,1},
    {0,1,1},{0,-1,-1},{0,1,-1},{0,-1,1},
    {1,1,1},{-1,-1,-1},{1,1,-1},{-1,-1,1},{1,-1,1},{-1,1,-1},{-1,1,1},{1,-1,-1}};

static double w1d(int c) { return c == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }

static int ipow(int b, int e) { int r = 1; while (e-- > 0) r *= b; return r; }

/* digit j of a packed order-n component index (first index fastest) */
static int digit(int idx, int j, int D) { return (idx / ipow(D, j)) % D; }

static double kdelta(int a, int b) { return a == b ? 1.0 : 0.0; }

/* Tensor Hermite polynomial component H^(n)_{a1..an}(xi), n <= 4, from the
 * Rodrigues formula of Sec. II.A written out order by order. */
static double hermite_comp(int n, const int *a, const double *x)
{
    switch (n) {
    case 0: return 1.0;
    case 1: return x[a[0]];
    case 2: return x[a[0]] * x[a[1]] - kdelta(a[0], a[1]);
    case 3:
        return x[a[0]] * x[a[1]] * x[a[2]]
             - x[a[0]] * kdelta(a[1], a[2]) - x[a[1]] * kdelta(a[0], a[2])
             - x[a[2]] * kdelta(a[0], a[1]);
    case 4:
        return x[a[0]] * x[a[1]] * x[a[2]] * x[a[3]]
             - x[a[0]] * x[a[1]] * kdelta(a[2], a[3])
             - x[a[0]] * x[a[2]] * kdelta(a[1], a[3])
             - x[a[0]] * x[a[3]] * kdelta(a[1], a[2])
             - x[a[1]] * x[a[2]] * kdelta(a[0], a[3])
             - x[a[1]] * x[a[3]] * kdelta(a[0], a[2])
             - x[a[2]] * x[a[3]] * kdelta(a[0], a[1])
             + kdelta(a[0], a[1]) * kdelta(a[2], a[3])
             + kdelta(a[0], a[2]) * kdelta(a[1], a[3])
             + kdelta(a[0], a[3]) * kdelta(a[1], a[2]);
    }
    return 0.0;
}

/* Is the component with index tuple a (order n) part of the retained set? */
static int retained(int id, int D, int n, const int *a)
{
    int m[3] = {0, 0, 0};
    for (int j = 0; j < n; ++j) m[a[j]]++;
    (void)D;
    if (id == OR_D2Q9 || id == OR_D3Q27)
        return m[0] <= 2 && m[1] <= 2 && m[2] <= 2;
    /* D3Q19 */
    if (n <= 2) return 1;
    int twos = 0, ones = 0;
    for (int k = 0; k < 3; ++k) { twos += m[k] == 2; ones += m[k] == 1; }
    if (n == 3) return twos == 1 && ones == 1;
    return 0;
}

static void lattice_init(int id, or_lattice *L)
{
    memset(L, 0, sizeof(*L));
    L->id = id;
    if (id == OR_D2Q9) {
        L->D = 2; L->Q = 9;
        for (int i = 0; i < 9; ++i) {
            for (int k = 0; k < 3; ++k) L->c[i][k] = C2Q9[i][k];
            L->w[i] = w1d(C2Q9[i][0]) * w1d(C2Q9[i][1]);
        }
    } else {
        L->D = 3; L->Q = (id == OR_D3Q19) ? 19 : 27;
        for (int i = 0; i < L->Q; ++i)
            for (int k = 0; k < 3; ++k) L->c[i][k] = C3Q27[i][k];
        if (id == OR_D3Q27) {
            for (int i = 0; i < 27; ++i)
                L->w[i] = w1d(L->c[i][0]) * w1d(L->c[i][1]) * w1d(L->c[i][2]);
        } else {
            /* D3Q19 rule: rest 1/3, faces 1/18, edges 1/36 */
            for (int i = 0; i < 19; ++i) {
                int nz = (L->c[i][0] != 0) + (L->c[i][1] != 0) + (L->c[i][2] != 0);
                L->w[i] = nz == 0 ? 1.0 / 3.0 : (nz == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
            }
        }
    }
    for (int i = 0; i < L->Q; ++i) {
        for (int k = 0; k < 3; ++k) L->xi[i][k] = SQ3 * L->c[i][k];
        for (int j = 0; j < L->Q; ++j)
            if (L->c[j][0] == -L->c[i][0] && L->c[j][1] == -L->c[i][1] &&
                L->c[j][2] == -L->c[i][2])
                L->opp[i] = j;
    }
    L->off[0] = 0;
    for (int n = 0; n <= OR_MAXN; ++n) L->off[n + 1] = L->off[n] + ipow(L->D, n);
    for (int n = 0; n <= OR_MAXN; ++n)
        for (int idx = 0; idx < ipow(L->D, n); ++idx) {
            int a[4];
            const int k = L->off[n] + idx;
            for (int j = 0; j < n; ++j) a[j] = digit(idx, j, L->D);
            L->order[k] = n;
            for (int j = 0; j < 4; ++j) L->dig[k][j] = j < n ? a[j] : 0;
            for (int S = 0; S < (1 << n); ++S) {
                int r = 0, m = 0, scale = 1;
                for (int j = 0; j < n; ++j)
                    if (!(S & (1 << j))) { r += a[j] * scale; scale *= L->D; ++m; }
                L->rest[k][S] = L->off[m] + r;
            }
            L->keep[L->off[n] + idx] = (unsigned char)retained(id, L->D, n, a);
            for (int i = 0; i < L->Q; ++i)
                L->H[i][L->off[n] + idx] = hermite_comp(n, a, L->xi[i]);
        }
}

/* ------------------------------------------------------------------------ */
/* Moment-space primitives (all tensors full and packed, Hermite units)     */
/* ------------------------------------------------------------------------ */

/* Eq. (dft), first line: a^(n) = sum_i f_i H^(n)(xi_i), n = 0..4 */
static void project(const or_lattice *L, const double *f, double *a)
{
    for (int k = 0; k < L->off[OR_MAXN + 1]; ++k) {
        double s = 0.0;
        for (int i = 0; i < L->Q; ++i) s += f[i] * L->H[i][k];
        a[k] = s;
    }
}

/* Eq. (dft), second line restricted to the retained components:
 * f_i = w_i sum_n (1/n!) A^(n) : H^(n)(xi_i), full contraction. */
static void reconstruct(const or_lattice *L, const double *A, double *f)
{
    static const double invfact[5] = {1.0, 1.0, 0.5, 1.0 / 6.0, 1.0 / 24.0};
    for (int i = 0; i < L->Q; ++i) {
        double s = 0.0;
        for (int n = 0; n <= OR_MAXN; ++n) {
            double sn = 0.0;
            for (int k = L->off[n]; k < L->off[n + 1]; ++k)
                if (L->keep[k]) sn += A[k] * L->H[i][k];
            s += invfact[n] * sn;
        }
        f[i] = L->w[i] * s;
    }
}

/* Equilibrium Hermite coefficients at theta = 1: a_0^(n) = rho u^{(x)n} */
static void equilibrium_moments(const or_lattice *L, double rho, const double *u, double *a0)
{
    for (int k = 0; k < L->off[OR_MAXN + 1]; ++k) {
        double p = rho;
        for (int j = 0; j < L->order[k]; ++j) p *= u[L->dig[k][j]];
        a0[k] = p;
    }
}

/* Frame shift by the vector s (Hermite addition theorem at theta = 1):
 *   out^(n)_{a1..an} = sum over subsets S of positions {1..n} of
 *                      prod_{j in S} s_{aj} * in^(n-|S|)_{a restricted to not-S}
 * i.e. out^(n) = sum_k C(n,k) s^k in^(n-k), the binomial coefficient counting
 * the distinct placements of the symmetric product.  s = -u maps raw moments
 * to central (co-moving) moments, s = +u maps back (Eq. bbd1). */
static void shift(const or_lattice *L, const double *s, const double *in, double *out)
{
    for (int k = 0; k < L->off[OR_MAXN + 1]; ++k) {
        const int n = L->order[k];
        double acc = 0.0;
        for (int S = 0; S < (1 << n); ++S) {
            double p = 1.0;
            for (int j = 0; j < n; ++j)
                if (S & (1 << j)) p *= s[L->dig[k][j]];
            acc += p * in[L->rest[k][S]];
        }
        out[k] = acc;
    }
}

/* ------------------------------------------------------------------------ */
/* Collision at one node.  The state is stored as deviations from the rest  */
/* weights, delta_i = fbar_i - w_i (fbar: the variable of Eq. newf), in     */
/* FP64: an O(1) population carries a rounding error of ~1e-17 per step,    */
/* which at a slowly decaying steady state leaves a floor of ~5e-12 on a    */
/* small velocity; the deviation carries it on its own, much smaller, size. */
/* The algebra is unchanged: the weights' Hermite coefficients are          */
/* (1, 0, 0, ...), so every moment of order >= 1 of fbar equals that of     */
/* delta, a^(0) = 1 + sum delta, and reconstructing a coefficient vector    */
/* with its order-0 entry lowered by one yields fbar_p - w directly.        */
/* gL: body-force acceleration in lattice units.  When dbg != NULL the      */
/* packed vectors [a_bar | a_0 | a_1 | d_1 | d_p | a_p] (6 x OR_PACK) are   */
/* written for tests.                                                       */
/* ------------------------------------------------------------------------ */
static void macroscopic(const or_lattice *L, const double *dev, const double *gL,
                        double *drho_out, double *rho_out, double *uH, double *gH)
{
    double drho = 0.0, j[3] = {0, 0, 0};
    for (int i = 0; i < L->Q; ++i) {
        drho += dev[i];
        for (int k = 0; k < L->D; ++k) j[k] += dev[i] * L->xi[i][k];
    }
    const double rho = 1.0 + drho;
    for (int k = 0; k < 3; ++k) { gH[k] = 0.0; uH[k] = 0.0; }
    for (int k = 0; k < L->D; ++k) {
        gH[k] = SQ3 * gL[k];
        /* Eq. (half_F): u = u_bar + F/(2 rho) with F = rho g */
        uH[k] = j[k] / rho + 0.5 * gH[k];
    }
    *drho_out = drho;
    *rho_out = rho;
}

/* Second-order equilibrium of the BGK section, minus w_i:
 * f_eq - w = w_i [ (rho - 1) + rho (xi.u + ((xi.u)^2 - u^2)/2) ] */
static double feq2_dev(const or_lattice *L, int i, double drho, double rho, const double *u)
{
    double xu = 0.0, uu = 0.0;
    for (int k = 0; k < L->D; ++k) { xu += L->xi[i][k] * u[k]; uu += u[k] * u[k]; }
    return L->w[i] * (drho + rho * (xu + 0.5 * (xu * xu - uu)));
}

static double force2(const or_lattice *L, int i, double rho, const double *u, const double *g)
{
    double gx = 0.0, gu = 0.0, ux = 0.0;
    for (int k = 0; k < L->D; ++k) {
        gx += g[k] * L->xi[i][k];
        gu += g[k] * u[k];
        ux += u[k] * L->xi[i][k];
    }
    /* F(xi) = rho omega [ g.(xi - u) + (g.xi)(u.xi) ],  F_i = w_i F / omega */
    return rho * L->w[i] * ((gx - gu) + gx * ux);
}

static void collide_bgk(const or_lattice *L, const double *tau, const double *dev,
                        const double *gL, double *dp)
{
    double drho, rho, u[3], g[3];
    macroscopic(L, dev, gL, &drho, &rho, u, g);
    const double th = tau[2];
    for (int i = 0; i < L->Q; ++i) {
        /* Eq. (explict_eq), with w_i subtracted from fbar and f_eq alike */
        dp[i] = dev[i] - (dev[i] - feq2_dev(L, i, drho, rho, u)) / th
              + (1.0 - 0.5 / th) * force2(L, i, rho, u, g);
    }
}

/* Order-n force coefficients in the co-moving frame, d_F^(n) = n g d^(n-1)
 * (the definition after Eq. Frc at theta = 1): the symmetric product of g
 * and d^(n-1) summed over the n positions g can take. */
static void force_order(const or_lattice *L, int n, const double *g, const double *d, double *dF)
{
    for (int k = L->off[n]; k < L->off[n + 1]; ++k) {
        double acc = 0.0;
        for (int j = 0; j < n; ++j) acc += g[L->dig[k][j]] * d[L->rest[k][1 << j]];
        dF[k] = acc;
    }
}

/* The second-order block with its traceless (shear) and trace (bulk) parts
 * scaled separately, Eq. (domg) with tau_{2,2} and tau_{2,0}:
 *   out = cs (X - delta tr(X)/D) + cb delta tr(X)/D
 *       = cs X + (cb - cs) delta tr(X)/D. */
static void split_order2(const or_lattice *L, double cs, double cb, const double *X, double *out)
{
    const int o = L->off[2], D = L->D;
    double tr = 0.0;
    for (int a = 0; a < D; ++a) tr += X[o + a + a * D];
    tr /= D;
    for (int k = o; k < L->off[3]; ++k) {
        const double iso = L->dig[k][0] == L->dig[k][1] ? tr : 0.0;
        out[k] = cs * X[k] + (cb - cs) * iso;
    }
}

static void collide_smrt(const or_lattice *L, const double *tau, double tau_b, int fneq, const double *dev,
                         const double *gL, double *dpop, double *dbg)
{
    double X[OR_PACK];
    double drho, rho, u[3], g[3], mu[3];
    double abar[OR_PACK], a0[OR_PACK], a1[OR_PACK], d1[OR_PACK], dp[OR_PACK], ap[OR_PACK];
    double tot[OR_PACK], dF[OR_PACK], d[OR_PACK];
    const int P = L->off[OR_MAXN + 1];
    macroscopic(L, dev, gL, &drho, &rho, u, g);
    for (int k = 0; k < 3; ++k) mu[k] = -u[k];

    project(L, dev, abar);                  /* Eq. (dft); orders >= 1 of fbar */
    abar[0] = rho;
    equilibrium_moments(L, rho, u, a0);     /* a_0^(n) = rho u^n */
    /* non-equilibrium raw moments a_bar_1 = a_bar - a_0; a_bar_1^(0) = 0 and
     * a_bar_1^(1) = -F/2 follow from the same subtraction (Eq. half_F). */
    for (int k = 0; k < P; ++k) a1[k] = abar[k] - a0[k];
    a1[0] = 0.0;
    shift(L, mu, a1, d1);                   /* RM -> RCM */
    /* force coefficients.  d_F^(1) = rho g always.  With the non-equilibrium
     * contributions, d_F^(n) = n g d^(n-1) needs the central moments d of f
     * (not fbar): d^(0) = rho, d^(1) = 0 (mass and momentum), and for n >= 2
     * Eq. (newf) in moment form, d_1bar^(n) = (tau_n/(tau_n - 1/2)) d^(n)
     * - d_F^(n)/2 with tau_n the tau-hat of the update, inverts to
     * d^(n) = (1 - 1/(2 tau_n)) (d_1bar^(n) + d_F^(n)/2).  Each order needs
     * only the one below it. */
    for (int k = 0; k < P; ++k) { dF[k] = 0.0; d[k] = 0.0; }
    d[0] = rho;
    for (int k = 0; k < L->D; ++k) dF[L->off[1] + k] = rho * g[k];
    if (fneq) {
        for (int n = 2; n <= OR_MAXN; ++n) {
            force_order(L, n, g, d, dF);
            for (int k = L->off[n]; k < L->off[n + 1]; ++k) X[k] = d1[k] + 0.5 * dF[k];
            if (n == 2) {
                split_order2(L, 1.0 - 0.5 / tau[2], 1.0 - 0.5 / tau_b, X, d);
            } else {
                for (int k = L->off[n]; k < L->off[n + 1]; ++k) d[k] = (1.0 - 0.5 / tau[n]) * X[k];
            }
        }
    }
    /* relaxation with the force, order by order (Eq. RHS, explicit form):
     * d_p^(n) = (1 - 1/tau_n) d_1^(n) + (1 - 1/(2 tau_n)) d_F^(n), d_p^(0) = 0,
     * the second order per traceless part (shear tau[2], bulk tau_b) */
    dp[0] = 0.0;
    for (int n = 1; n <= OR_MAXN; ++n) {
        const double t = tau[n];
        for (int k = L->off[n]; k < L->off[n + 1]; ++k)
            dp[k] = (1.0 - 1.0 / t) * d1[k] + (1.0 - 0.5 / t) * dF[k];
    }
    {
        double r1[OR_PACK], r2[OR_PACK];
        split_order2(L, 1.0 - 1.0 / tau[2], 1.0 - 1.0 / tau_b, d1, r1);
        split_order2(L, 1.0 - 0.5 / tau[2], 1.0 - 0.5 / tau_b, dF, r2);
        for (int k = L->off[2]; k < L->off[3]; ++k) dp[k] = r1[k] + r2[k];
    }
    shift(L, u, dp, ap);                    /* RCM -> RM (Eq. bbd1) */
    for (int k = 0; k < P; ++k) tot[k] = a0[k] + ap[k];
    tot[0] = drho;                          /* rho - 1: reconstruct fbar_p - w */
    reconstruct(L, tot, dpop);              /* post-collision reconstruction */
    if (dbg) {
        memcpy(dbg + 0 * OR_PACK, abar, sizeof(double) * P);
        memcpy(dbg + 1 * OR_PACK, a0, sizeof(double) * P);
        memcpy(dbg + 2 * OR_PACK, a1, sizeof(double) * P);
        memcpy(dbg + 3 * OR_PACK, d1, sizeof(double) * P);
        memcpy(dbg + 4 * OR_PACK, dp, sizeof(double) * P);
        memcpy(dbg + 5 * OR_PACK, ap, sizeof(double) * P);
    }
}

/* Raw-moment MRT of the appendix, at theta = 1 (u_1 = u_2 = u u):
 *   a_p^(n) = a_0^(n) + (1 - 1/tau_n) a_1bar^(n) + (1 - 1/(2 tau_n)) a_F^(n),
 * with a_1bar^(1) = -F/2, a_1bar^(2), a_1bar^(3) projected, the fourth order
 * from the recursion
 *   a_1bar^(4) = 4 u a_1bar^(3) - 6 u u a_1bar^(2) + 4 u u u a_1bar^(1)
 * (each term summed over the distinct placements of the u's), and the
 * force's equilibrium part a_F^(n) = n F u^(n-1) (placements of F among the
 * n indices, u at the others). */
static void collide_mrt_raw(const or_lattice *L, const double *tau, const double *dev,
                            const double *gL, double *dpop)
{
    double drho, rho, u[3], g[3];
    double abar[OR_PACK], a0[OR_PACK], a1[OR_PACK], aF[OR_PACK], tot[OR_PACK];
    const int P = L->off[OR_MAXN + 1];
    macroscopic(L, dev, gL, &drho, &rho, u, g);
    project(L, dev, abar);
    abar[0] = rho;
    equilibrium_moments(L, rho, u, a0);
    for (int k = 0; k < P; ++k) a1[k] = abar[k] - a0[k];
    a1[0] = 0.0;
    for (int k = 0; k < L->D; ++k) a1[L->off[1] + k] = -0.5 * rho * g[k];
    for (int k = L->off[4]; k < L->off[5]; ++k) {
        double acc = 0.0;
        for (int S = 1; S < 15; ++S) {          /* non-empty proper subsets of the 4 positions */
            int m = 0;
            double p = 1.0;
            for (int j = 0; j < 4; ++j)
                if (S & (1 << j)) { p *= u[L->dig[k][j]]; ++m; }
            acc += (m == 2 ? -1.0 : 1.0) * p * a1[L->rest[k][S]];
        }
        a1[k] = acc;
    }
    for (int k = 0; k < P; ++k) {
        const int n = L->order[k];
        double acc = 0.0;
        for (int j = 0; j < n; ++j) {
            double p = rho * g[L->dig[k][j]];
            for (int i = 0; i < n; ++i)
                if (i != j) p *= u[L->dig[k][i]];
            acc += p;
        }
        aF[k] = acc;
    }
    tot[0] = drho;                              /* rho - 1: reconstruct fbar_p - w */
    for (int k = 1; k < P; ++k) {
        const double t = tau[L->order[k]];
        tot[k] = a0[k] + (1.0 - 1.0 / t) * a1[k] + (1.0 - 0.5 / t) * aF[k];
    }
    reconstruct(L, tot, dpop);
}

/* delta = f_eq - F/2 - w with the collision model's own equilibrium and force */
static void initial_node(const or_lattice *L, int collision, double rho, const double *uL,
                         const double *gL, double *dev)
{
    double u[3] = {0, 0, 0}, g[3] = {0, 0, 0};
    const double drho = rho - 1.0;
    for (int k = 0; k < L->D; ++k) { u[k] = SQ3 * uL[k]; g[k] = SQ3 * gL[k]; }
    if (collision == OR_BGK) {
        for (int i = 0; i < L->Q; ++i)
            dev[i] = feq2_dev(L, i, drho, rho, u) - 0.5 * force2(L, i, rho, u, g);
        return;
    }
    double a0[OR_PACK], dF[OR_PACK], aF[OR_PACK], A[OR_PACK];
    const int P = L->off[OR_MAXN + 1];
    equilibrium_moments(L, rho, u, a0);
    for (int k = 0; k < P; ++k) dF[k] = 0.0;
    for (int k = 0; k < L->D; ++k) dF[L->off[1] + k] = rho * g[k];
    shift(L, u, dF, aF); /* raw-moment force coefficients a_F^(n) = n F u^(n-1) */
    for (int k = 0; k < P; ++k) A[k] = a0[k] - 0.5 * aF[k];
    A[0] = drho;
    reconstruct(L, A, dev);
}

/* ------------------------------------------------------------------------ */
/* Public interface (ctypes).  Fields are SoA: f[i][z][y][x], u[a][z][y][x], */
/* g[a][z][y][x]; solid is one byte per node (nullable).                     */
/* ------------------------------------------------------------------------ */
typedef struct {
    int lattice, collision;
    int nx, ny, nz;
    int periodic[3];
    double tau[5];
    double tau_bulk;  /* tau_{2,0} of the SMRT forms; <= 0 means tau[2] */
} or_params;

static int check_params(const or_params *p, or_lattice *L)
{
    if (p->lattice < 0 || p->lattice > 2 || p->collision < 0 || p->collision > 3) return -1;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return -1;
    lattice_init(p->lattice, L);
    if (L->D == 2 && p->nz != 1) return -1;
    if (p->collision == OR_BGK && !(p->tau[2] > 0.5)) return -1;
    if (p->tau_bulk > 0.0 && p->tau_bulk != p->tau[2] &&
        !(p->collision == OR_SMRT || p->collision == OR_SMRT_FNEQ))
        return -1;
    if (p->tau_bulk > 0.0 && !(p->tau_bulk > 0.5)) return -1;
    if (p->collision != OR_BGK)
        for (int n = 2; n <= 4; ++n)
            if (!(p->tau[n] > 0.5)) return -1;
    return 0;
}

int or_lattice_tables(int lattice, int *D, int *Q, int *c, double *w, int *opp)
{
    or_lattice L;
    if (lattice < 0 || lattice > 2) return -1;
    lattice_init(lattice, &L);
    *D = L.D; *Q = L.Q;
    for (int i = 0; i < L.Q; ++i) {
        for (int k = 0; k < 3; ++k) c[3 * i + k] = L.c[i][k];
        w[i] = L.w[i];
        opp[i] = L.opp[i];
    }
    return 0;
}

/* Hermite table H^(n)(xi_i) (Q x 121 packed, zero-padded for D = 2) and the
 * retained mask (121 bytes); for tests of orthogonality and the transform. */
int or_hermite_table(int lattice, double *H, unsigned char *keep, int *off)
{
    or_lattice L;
    if (lattice < 0 || lattice > 2) return -1;
    lattice_init(lattice, &L);
    for (int i = 0; i < L.Q; ++i)
        for (int k = 0; k < OR_PACK; ++k) H[i * OR_PACK + k] = L.H[i][k];
    for (int k = 0; k < OR_PACK; ++k) keep[k] = L.keep[k];
    for (int n = 0; n <= OR_MAXN + 1; ++n) off[n] = L.off[n];
    return 0;
}

/* Hermite polynomial of an arbitrary argument (packed n = 0..4). */
int or_hermite_at(int D, const double *x, double *H)
{
    int o = 0;
    for (int n = 0; n <= OR_MAXN; ++n)
        for (int idx = 0; idx < ipow(D, n); ++idx) {
            int a[4];
            for (int j = 0; j < n; ++j) a[j] = digit(idx, j, D);
            H[o++] = hermite_comp(n, a, x);
        }
    return o;
}

int or_project(int lattice, const double *f, double *a)
{
    or_lattice L;
    if (lattice < 0 || lattice > 2) return -1;
    lattice_init(lattice, &L);
    project(&L, f, a);
    return 0;
}

int or_reconstruct(int lattice, const double *A, double *f)
{
    or_lattice L;
    if (lattice < 0 || lattice > 2) return -1;
    lattice_init(lattice, &L);
    reconstruct(&L, A, f);
    return 0;
}

int or_shift(int lattice, const double *s, const double *in, double *out)
{
    or_lattice L;
    if (lattice < 0 || lattice > 2) return -1;
    lattice_init(lattice, &L);
    shift(&L, s, in, out);
    return 0;
}

/* One node's collision (lattice-unit g) on populations fbar -> fbar_p.
 * dbg: 6 x 121 doubles or NULL. */
int or_collide_node(const or_params *p, const double *fbar, const double *gL, double *fp,
                    double *dbg)
{
    or_lattice L;
    double dev[OR_MAXQ], dp[OR_MAXQ];
    if (check_params(p, &L)) return -1;
    for (int i = 0; i < L.Q; ++i) dev[i] = fbar[i] - L.w[i];
    if (p->collision == OR_BGK) collide_bgk(&L, p->tau, dev, gL, dp);
    else if (p->collision == OR_MRT_RAW) collide_mrt_raw(&L, p->tau, dev, gL, dp);
    else collide_smrt(&L, p->tau, p->tau_bulk > 0.0 ? p->tau_bulk : p->tau[2], p->collision == OR_SMRT_FNEQ,
                      dev, gL, dp, dbg);
    for (int i = 0; i < L.Q; ++i) fp[i] = L.w[i] + dp[i];
    return 0;
}

/* Initial populations fbar at one node (lattice units). */
int or_initial_node(const or_params *p, double rho, const double *uL, const double *gL, double *f)
{
    or_lattice L;
    double dev[OR_MAXQ];
    if (check_params(p, &L)) return -1;
    initial_node(&L, p->collision, rho, uL, gL, dev);
    for (int i = 0; i < L.Q; ++i) f[i] = L.w[i] + dev[i];
    return 0;
}

static size_t n_nodes(const or_params *p) { return (size_t)p->nx * p->ny * p->nz; }

/* State arrays hold deviations delta = fbar - w, [Q][N].
 * delta = f_eq(rho0, u0) - F/2 - w at fluid nodes, 0 at solid nodes.
 * rho0 / u0 nullable (=> 1 / 0). */
int or_init(const or_params *p, const unsigned char *solid, const double *rho0,
            const double *u0, const double *g, double *f)
{
    or_lattice L;
    if (check_params(p, &L)) return -1;
    const size_t N = n_nodes(p);
    for (size_t x = 0; x < N; ++x) {
        double fl[OR_MAXQ], uL[3] = {0, 0, 0}, gL[3] = {0, 0, 0};
        if (solid && solid[x]) {
            for (int i = 0; i < L.Q; ++i) f[(size_t)i * N + x] = 0.0;
            continue;
        }
        for (int k = 0; k < L.D; ++k) {
            uL[k] = u0 ? u0[(size_t)k * N + x] : 0.0;
            gL[k] = g ? g[(size_t)k * N + x] : 0.0;
        }
        initial_node(&L, p->collision, rho0 ? rho0[x] : 1.0, uL, gL, fl);
        for (int i = 0; i < L.Q; ++i) f[(size_t)i * N + x] = fl[i];
    }
    return 0;
}

/* One time step: collide every fluid node, then stream (push) with periodic
 * wrap or halfway bounce-back (Sec. II.C: f_i(x + xi_i, t+1) = fbar_{i,p}(x,t)).
 * f_in and f_out must not alias. */
int or_step(const or_params *p, const unsigned char *solid, const double *g,
            const double *f_in, double *f_out)
{
    or_lattice L;
    if (check_params(p, &L)) return -1;
    const size_t N = n_nodes(p);
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    for (int i = 0; i < L.Q; ++i)
        for (size_t x = 0; x < N; ++x) f_out[(size_t)i * N + x] = 0.0;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (long long xl = 0; xl < (long long)N; ++xl) {
        const size_t x = (size_t)xl;
        if (solid && solid[x]) continue;
        double fb[OR_MAXQ], fp[OR_MAXQ], gL[3] = {0, 0, 0};
        for (int i = 0; i < L.Q; ++i) fb[i] = f_in[(size_t)i * N + x];
        for (int k = 0; k < L.D; ++k) gL[k] = g ? g[(size_t)k * N + x] : 0.0;
        if (p->collision == OR_BGK) collide_bgk(&L, p->tau, fb, gL, fp);
        else if (p->collision == OR_MRT_RAW) collide_mrt_raw(&L, p->tau, fb, gL, fp);
        else collide_smrt(&L, p->tau, p->tau_bulk > 0.0 ? p->tau_bulk : p->tau[2],
                          p->collision == OR_SMRT_FNEQ, fb, gL, fp, NULL);
        const int X = (int)(x % nx), Y = (int)((x / nx) % ny), Z = (int)(x / ((size_t)nx * ny));
        for (int i = 0; i < L.Q; ++i) {
            int t[3] = {X + L.c[i][0], Y + L.c[i][1], Z + L.c[i][2]};
            const int n3[3] = {nx, ny, nz};
            int wall = 0;
            for (int k = 0; k < 3; ++k) {
                if (t[k] < 0 || t[k] >= n3[k]) {
                    if (p->periodic[k]) t[k] = (t[k] + n3[k]) % n3[k];
                    else wall = 1;
                }
            }
            size_t y = 0;
            if (!wall) {
                y = ((size_t)t[2] * ny + t[1]) * nx + t[0];
                if (solid && solid[y]) wall = 1;
            }
            if (wall) f_out[(size_t)L.opp[i] * N + x] = fp[i]; /* halfway bounce-back */
            else f_out[(size_t)i * N + y] = fp[i];
        }
    }
    return 0;
}

/* rho, u (lattice units, physical half-shifted velocity) and the totals
 * [M, Px, Py, Pz] summed serially over fluid nodes.  Solid nodes report
 * rho = 1, u = 0 and are left out of the totals.  Outputs nullable. */
int or_moments(const or_params *p, const unsigned char *solid, const double *g,
               const double *f, double *rho, double *u, double *totals)
{
    or_lattice L;
    if (check_params(p, &L)) return -1;
    const size_t N = n_nodes(p);
    double T[4] = {0, 0, 0, 0};
    for (size_t x = 0; x < N; ++x) {
        double r = 0.0, dr = 0.0, j[3] = {0, 0, 0}, uu[3] = {0, 0, 0};
        int s = solid && solid[x];
        if (!s) {
            for (int i = 0; i < L.Q; ++i) {
                double di = f[(size_t)i * N + x];
                dr += di;
                for (int k = 0; k < L.D; ++k) j[k] += di * L.c[i][k];
            }
            r = 1.0 + dr;
            for (int k = 0; k < L.D; ++k) {
                double gk = g ? g[(size_t)k * N + x] : 0.0;
                uu[k] = j[k] / r + 0.5 * gk; /* Eq. (half_F) in lattice units */
            }
            T[0] += r;
            for (int k = 0; k < L.D; ++k) T[1 + k] += r * uu[k];
        } else {
            r = 1.0;
        }
        if (rho) rho[x] = r;
        if (u)
            for (int k = 0; k < L.D; ++k) u[(size_t)k * N + x] = uu[k];
    }
    if (totals)
        for (int k = 0; k < 4; ++k) totals[k] = T[k];
    return 0;
}

/* Round a double to a narrower binary format, round-to-nearest-even, with
 * gradual underflow and overflow to infinity.  mant = stored mantissa bits,
 * emin = exponent of the smallest normal, maxv = largest finite value. */
static double round_format(double x, int mant, int emin, double maxv)
{
    if (x == 0.0 || !isfinite(x)) return x;
    int e;
    frexp(x, &e);              /* |x| in [2^(e-1), 2^e) */
    int lead = e - 1;
    if (lead < emin) lead = emin;
    const double q = ldexp(1.0, lead - mant); /* spacing of the format near x */
    const double r = nearbyint(x / q) * q;    /* ties to even under FE_TONEAREST */
    if (fabs(r) > maxv) return copysign(INFINITY, x);
    return r;
}

/* Storage-precision emulation: mode 1 = FP32, 2 = FP16, 3 = BF16 applied to
 * the stored deviations delta_i = fbar_i - w_i (solid nodes included). */
int or_round_storage(const or_params *p, int mode, double *f)
{
    or_lattice L;
    if (check_params(p, &L)) return -1;
    const size_t N = n_nodes(p);
    for (int i = 0; i < L.Q; ++i)
        for (size_t x = 0; x < N; ++x) {
            double d = f[(size_t)i * N + x];
            switch (mode) {
            case 1: d = round_format(d, 23, -126, 3.4028234663852886e38); break;
            case 2: d = round_format(d, 10, -14, 65504.0); break;
            case 3: d = round_format(d, 7, -126, 3.3895313892515355e38); break;
            default: break;
            }
            f[(size_t)i * N + x] = d;
        }
    return 0;
}

int or_round_value(int mode, const double *x, double *y, int n)
{
    for (int k = 0; k < n; ++k) {
        switch (mode) {
        case 1: y[k] = round_format(x[k], 23, -126, 3.4028234663852886e38); break;
        case 2: y[k] = round_format(x[k], 10, -14, 65504.0); break;
        case 3: y[k] = round_format(x[k], 7, -126, 3.3895313892515355e38); break;
        default: y[k] = x[k];
        }
    }
    return 0;
}

/* Run nsteps steps with a time-independent force field; ping-pongs between
 * f and a caller-provided work buffer; result ends in f. */
int or_run(const or_params *p, const unsigned char *solid, const double *g, double *f,
           double *work, long long nsteps, int round_mode)
{
    or_lattice L;
    if (check_params(p, &L)) return -1;
    const size_t NQ = n_nodes(p) * (size_t)L.Q;
    for (long long s = 0; s < nsteps; ++s) {
        if (or_step(p, solid, g, f, work)) return -1;
        if (round_mode) or_round_storage(p, round_mode, work);
        memcpy(f, work, NQ * sizeof(double));
    }
    return 0;
}

int or_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
