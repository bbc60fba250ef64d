/*
 * Plain, slow, single-threaded CPU oracle for three-precision GADI.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
 * its Python binding) may link, load or call this file; only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark use it.  It shares no
 * code, header, table or constant generator with the CUDA path.
 *
 * What it computes (arXiv 2512.21164):
 *   - the splitting A = M + N with H = alpha I + M and S = alpha I + N
 *     (Sec. 3.1, "eq:split"), for the HSS choice M = (A + A^T)/2 and
 *     N = (A - A^T)/2 used for every problem of Sec. 5;
 *   - Algorithm 1 (mixed precision GADI): r = b - A x in u_r, solve
 *     (alpha I + M) z = r in u_s, solve (alpha I + N) y = (2 - omega) alpha z in
 *     u_s, x = x + y in u;
 *   - the inner solvers of Sec. 5.1: CG on the SPD shifted part H and CG on the
 *     normal equations S^T S y = S^T g for the shifted skew part S.
 *
 * Precision model (Sec. 5.1 "GADI-FP32" / "GADI-BF16", Table 1):
 *   u = u_r = FP64 always.  u_s is FP64, FP32, or BF16 storage with FP32
 *   arithmetic.  Every stored inner vector element is rounded to u_s at each
 *   write: r_s, the CG vectors r, p, z, the CGNR vectors t, p, y, the scaled
 *   right-hand side g and the intermediate S p of CGNR.  The products H p and
 *   S^T (S p), consumed where they are formed, are carried in the compute
 *   type (double for FP64, float otherwise).  An FP32 dot product is the
 *   float nearest to the exact dot product of the stored vectors (the FP32
 *   result a summation tree approaches; sequential FP32 accumulation would
 *   add an order-dependent error of up to m u).
 *   FP32 arithmetic is C float arithmetic (IEEE binary32, round to nearest
 *   even; build with -ffp-contract=off so no fused multiply-add is formed).
 *   FP64 operator products are accumulated with C99 fma() (one rounding per
 *   neighbour term, in the fixed order below), as are the FP64 CG updates.
 *   BF16 rounding is written out from its definition: round to nearest, ties
 *   to even, at 8 significant bits with the binary32 exponent range.
 *
 * Operator layout: a grid nx x ny (x nz) in row-major order, x fastest.  The
 * stencils are the centred finite-difference discretisations of Sec. 5.2-5.4,
 * scaled by h^2 so that entries are O(1).  A general operator is written as
 *   (Op v)_i = d v_i + sum_dir c_dir v_nbr(i,dir)  [+ i e v_i  for complex]
 * with neighbours W,E (x-1,x+1), S,N (y-1,y+1), B,T (z-1,z+1) and zero
 * Dirichlet values outside the grid.  Sums are taken in that fixed order.
 * Complex vectors are interleaved (re, im) pairs.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Parallel loops for the all-core build of the timed CPU baseline (built with
 * -fopenmp into a second library).  The default build, the one every parity
 * test uses, is compiled without OpenMP: these expand to nothing and every
 * loop and sum runs sequentially in index order.  In the OpenMP build the
 * sums are split by thread, which changes only their rounding order. */
#ifdef _OPENMP
#define ORC_PRAGMA(x) _Pragma(#x)
#define OMP_FOR ORC_PRAGMA(omp parallel for schedule(static))
#define OMP_FOR_COLLAPSE2 ORC_PRAGMA(omp parallel for collapse(2) schedule(static))
#define OMP_FOR_SUM(v) ORC_PRAGMA(omp parallel for reduction(+ : v) schedule(static))
#else
#define OMP_FOR
#define OMP_FOR_COLLAPSE2
#define OMP_FOR_SUM(v)
#endif

/* ------------------------------------------------------------------------ */
/* precisions (u_s)                                                          */
/* ------------------------------------------------------------------------ */
enum { ORC_FP64 = 0, ORC_FP32 = 1, ORC_BF16 = 2 };

/* Round a double to the nearest BF16 value (ties to even), returned as a
 * double.  BF16: 8 significant bits, exponent range of binary32 (Table 1).
 * Normal numbers in [2^(e-1), 2^e) have spacing 2^(e-8); below 2^-126 the
 * spacing is fixed at 2^-133 (subnormals).  Overflow past the largest finite
 * value (2 - 2^-7) 2^127 by half a spacing or more gives infinity. */
double orc_round_bf16(double v)
{
    if (isnan(v)) return NAN;
    if (isinf(v) || v == 0.0) return v;
    int e;
    (void)frexp(v, &e); /* |v| = m 2^e with m in [0.5, 1) */
    int q = e - 8;
    if (q < -133) q = -133;
    double scaled = ldexp(v, -q);      /* exact: power-of-two scaling */
    double r = ldexp(rint(scaled), q); /* rint rounds half to even */
    const double maxbf = ldexp(255.0, 120); /* (2 - 2^-7) 2^127 */
    if (fabs(r) > maxbf) return v > 0 ? INFINITY : -INFINITY;
    return r;
}

double orc_round_fp32(double v) { return (double)(float)v; }

double orc_round(int prec, double v)
{
    if (prec == ORC_FP32) return orc_round_fp32(v);
    if (prec == ORC_BF16) return orc_round_bf16(v);
    return v;
}

/* Store a float that already carries FP32 arithmetic into u_s. */
static float st_f(int prec, float v)
{
    if (prec == ORC_BF16) return (float)orc_round_bf16((double)v);
    return v;
}

/* ------------------------------------------------------------------------ */
/* operators                                                                 */
/* ------------------------------------------------------------------------ */
enum { ORC_K_2D5 = 0, ORC_K_3D7 = 1, ORC_K_C2D5 = 2, ORC_K_CSR = 3 };
enum { OP_A = 0, OP_M = 1, OP_N = 2, OP_H = 3, OP_S = 4, OP_ST = 5 };

typedef struct {
    int kind;
    int nx, ny, nz;
    /* stencil coefficients: d, W, E, S, N, B, T and the imaginary diagonal e */
    double d, c[6], e;
    /* complex class with a per-point imaginary diagonal: e_i = ep[i] (null: e) */
    const double *ep;
    /* CSR (kind ORC_K_CSR): y = d*x + V x, V given in CSR */
    int n;
    const int *rowptr, *col;
    const double *val;
} orc_op;

/* Coefficients of A, M and N for the stencil problems.
 *   2D (Sec. 5.2 with the convection term beta . grad u and a reaction
 *   term kappa u, h^2-scaled): A = M + N with
 *     M: centre 4 + kappa, every neighbour -1 (the h^2-scaled 5-point
 *     Laplacian plus the reaction);
 *     N: E +c_x, W -c_x, N +c_y, S -c_y, with c_i = beta_i h / 2.
 *   3D (Sec. 5.3): the same with centre 6 + kappa and a third axis.
 *   complex (Sec. 5.4, W + iT with W = L + kappa I, T = sigma I):
 *     M = W (centre 4 + kappa, neighbours -1), N = i sigma I.
 * out: [0]=d, [1..6]=W,E,S,N,B,T, [7]=e for the requested part
 * (0 = A, 1 = M, 2 = N). */
void orc_stencil_coeffs(int kind, int part, double h, const double *beta,
                        double kappa, double sigma, double *out)
{
    double cx = beta[0] * h / 2.0, cy = beta[1] * h / 2.0, cz = beta[2] * h / 2.0;
    double Md = 0, Mc[6] = {0, 0, 0, 0, 0, 0}, Nc[6] = {0, 0, 0, 0, 0, 0}, Ne = 0;
    if (kind == ORC_K_2D5) {
        Md = 4.0 + kappa;
        Mc[0] = Mc[1] = Mc[2] = Mc[3] = -1.0;
        Nc[0] = -cx; Nc[1] = cx; Nc[2] = -cy; Nc[3] = cy;
    } else if (kind == ORC_K_3D7) {
        Md = 6.0 + kappa;
        for (int k = 0; k < 6; k++) Mc[k] = -1.0;
        Nc[0] = -cx; Nc[1] = cx; Nc[2] = -cy; Nc[3] = cy; Nc[4] = -cz; Nc[5] = cz;
    } else { /* complex 2D */
        Md = 4.0 + kappa;
        Mc[0] = Mc[1] = Mc[2] = Mc[3] = -1.0;
        Ne = sigma;
    }
    for (int k = 0; k < 8; k++) out[k] = 0.0;
    if (part == 0) {
        out[0] = Md;
        for (int k = 0; k < 6; k++) out[1 + k] = Mc[k] + Nc[k];
        out[7] = Ne;
    } else if (part == 1) {
        out[0] = Md;
        for (int k = 0; k < 6; k++) out[1 + k] = Mc[k];
    } else {
        for (int k = 0; k < 6; k++) out[1 + k] = Nc[k];
        out[7] = Ne;
    }
}

static int op_len(const orc_op *op)
{
    if (op->kind == ORC_K_CSR) return op->n;
    int n = op->nx * op->ny * (op->kind == ORC_K_3D7 ? op->nz : 1);
    return op->kind == ORC_K_C2D5 ? 2 * n : n;
}

/* neighbour index (point index, not element index) or -1 outside */
static long nbr(const orc_op *op, int ix, int iy, int iz, int dir)
{
    int nx = op->nx, ny = op->ny, nz = op->kind == ORC_K_3D7 ? op->nz : 1;
    switch (dir) {
    case 0: ix--; break;
    case 1: ix++; break;
    case 2: iy--; break;
    case 3: iy++; break;
    case 4: iz--; break;
    default: iz++; break;
    }
    if (ix < 0 || ix >= nx || iy < 0 || iy >= ny || iz < 0 || iz >= nz) return -1;
    return ((long)iz * ny + iy) * nx + ix;
}

/* y = Op x in double, fixed summation order, each neighbour term added
 * with a fused multiply-add: s = d x_i, then s = fma(c_dir, x_nbr, s). */
static void apply_d(const orc_op *op, const double *x, double *y)
{
    if (op->kind == ORC_K_CSR) {
        OMP_FOR
        for (int i = 0; i < op->n; i++) {
            double s = op->d * x[i];
            for (int k = op->rowptr[i]; k < op->rowptr[i + 1]; k++)
                s = fma(op->val[k], x[op->col[k]], s);
            y[i] = s;
        }
        return;
    }
    int nz = op->kind == ORC_K_3D7 ? op->nz : 1;
    int ndir = op->kind == ORC_K_3D7 ? 6 : 4;
    int cplx = op->kind == ORC_K_C2D5;
    OMP_FOR_COLLAPSE2
    for (int iz = 0; iz < nz; iz++)
        for (int iy = 0; iy < op->ny; iy++)
            for (int ix = 0; ix < op->nx; ix++) {
                long i = ((long)iz * op->ny + iy) * op->nx + ix;
                if (!cplx) {
                    double s = op->d * x[i];
                    for (int dir = 0; dir < ndir; dir++) {
                        long j = nbr(op, ix, iy, iz, dir);
                        if (j >= 0) s = fma(op->c[dir], x[j], s);
                    }
                    y[i] = s;
                } else {
                    double sr = op->d * x[2 * i], si = op->d * x[2 * i + 1];
                    for (int dir = 0; dir < ndir; dir++) {
                        long j = nbr(op, ix, iy, iz, dir);
                        if (j >= 0) {
                            sr = fma(op->c[dir], x[2 * j], sr);
                            si = fma(op->c[dir], x[2 * j + 1], si);
                        }
                    }
                    /* (i e) (xr + i xi) = -e xi + i e xr */
                    double ei = op->ep ? op->ep[i] : op->e;
                    sr = fma(-ei, x[2 * i + 1], sr);
                    si = fma(ei, x[2 * i], si);
                    y[2 * i] = sr;
                    y[2 * i + 1] = si;
                }
            }
}

/* The same in float arithmetic; coefficients are given already rounded to
 * u_s and converted to float. */
typedef struct {
    float d, c[6], e;
    const float *val; /* CSR values rounded to u_s */
    const float *ep;  /* per-point imaginary diagonal (null: e) */
} op_f;

static void apply_f(const orc_op *op, const op_f *cf, const float *x, float *y)
{
    if (op->kind == ORC_K_CSR) {
        OMP_FOR
        for (int i = 0; i < op->n; i++) {
            float s = cf->d * x[i];
            for (int k = op->rowptr[i]; k < op->rowptr[i + 1]; k++)
                s = s + cf->val[k] * x[op->col[k]];
            y[i] = s;
        }
        return;
    }
    int nz = op->kind == ORC_K_3D7 ? op->nz : 1;
    int ndir = op->kind == ORC_K_3D7 ? 6 : 4;
    int cplx = op->kind == ORC_K_C2D5;
    OMP_FOR_COLLAPSE2
    for (int iz = 0; iz < nz; iz++)
        for (int iy = 0; iy < op->ny; iy++)
            for (int ix = 0; ix < op->nx; ix++) {
                long i = ((long)iz * op->ny + iy) * op->nx + ix;
                if (!cplx) {
                    float s = cf->d * x[i];
                    for (int dir = 0; dir < ndir; dir++) {
                        long j = nbr(op, ix, iy, iz, dir);
                        if (j >= 0) s = s + cf->c[dir] * x[j];
                    }
                    y[i] = s;
                } else {
                    float sr = cf->d * x[2 * i], si = cf->d * x[2 * i + 1];
                    for (int dir = 0; dir < ndir; dir++) {
                        long j = nbr(op, ix, iy, iz, dir);
                        if (j >= 0) {
                            sr = sr + cf->c[dir] * x[2 * j];
                            si = si + cf->c[dir] * x[2 * j + 1];
                        }
                    }
                    float ei = cf->ep ? cf->ep[i] : cf->e;
                    sr = sr - ei * x[2 * i + 1];
                    si = si + ei * x[2 * i];
                    y[2 * i] = sr;
                    y[2 * i + 1] = si;
                }
            }
}

static orc_op make_stencil_op(int kind, int nx, int ny, int nz, const double *co)
{
    orc_op op;
    memset(&op, 0, sizeof op);
    op.kind = kind;
    op.nx = nx; op.ny = ny; op.nz = nz;
    op.d = co[0];
    for (int k = 0; k < 6; k++) op.c[k] = co[1 + k];
    op.e = co[7];
    return op;
}

/* Public: y = Op x in FP64 for a stencil operator with coefficients co[8]. */
void orc_stencil_apply(int kind, int nx, int ny, int nz, const double *co,
                       const double *x, double *y)
{
    orc_op op = make_stencil_op(kind, nx, ny, nz, co);
    apply_d(&op, x, y);
}

/* Public: y = (d I + V) x in FP64 for a CSR matrix V. */
void orc_csr_apply(int n, const int *rowptr, const int *col, const double *val,
                   double d, const double *x, double *y)
{
    orc_op op;
    memset(&op, 0, sizeof op);
    op.kind = ORC_K_CSR; op.n = n; op.rowptr = rowptr; op.col = col; op.val = val; op.d = d;
    apply_d(&op, x, y);
}

/* ------------------------------------------------------------------------ */
/* the GADI operator set for one solve                                       */
/* ------------------------------------------------------------------------ */
/* Everything the solve needs: A (FP64), and H, S, S^T in u_s.
 * Stencils: H = (alpha + d_M) I + M_offdiag, S = alpha I + N, S^T = alpha I - N
 * (N is skew: N^T = -N; in the complex case the adjoint S^H = alpha I - i sigma I
 * plays the role of S^T).  The stored coefficients of H and S are rounded to
 * u_s: H's diagonal as fl(alpha + d_M), as a stored matrix H would hold it
 * (Sec. 5.1, on the memory GADI needs).
 * CSR: M = (A + A^T)/2 and N = (A - A^T)/2 are passed in; H = alpha I + M,
 * S = alpha I + N and S^T = alpha I - N are formed in FP64 on M's pattern and
 * their values rounded to u_s. */
typedef struct {
    int prec;
    orc_op A;        /* FP64 */
    orc_op H, S, St; /* coefficient values in double, already rounded to u_s */
    /* float copies for FP32 / BF16 arithmetic */
    op_f Hf, Sf, Stf;
    float *Mval_f, *Nval_f, *NvalT_f;
    double *Mval_d, *Nval_d, *NvalT_d;
    /* per-point T of the complex class in u_s: S (+T), S^T (-T), double and float */
    double *es_d, *est_d;
    float *es_f, *est_f;
} gadi_ops;

static void fill_opf(const orc_op *o, op_f *f, const float *val)
{
    f->d = (float)o->d;
    for (int k = 0; k < 6; k++) f->c[k] = (float)o->c[k];
    f->e = (float)o->e;
    f->val = val;
    f->ep = NULL;
}

/* problem descriptor passed from Python as flat arguments */
typedef struct {
    int kind, nx, ny, nz;
    double h, beta[3], kappa, sigma;
    int n;
    const int *rowptr, *col;
    const double *aval;       /* A  */
    const int *mrowptr, *mcol; /* M = (A + A^T)/2 pattern; N shares it */
    const double *mval, *nval;
    const double *sigma_pt; /* complex class: per-point T (nx*ny values) or null */
} orc_problem;

static int build_ops(const orc_problem *p, double alpha, int prec, gadi_ops *g)
{
    memset(g, 0, sizeof *g);
    g->prec = prec;
    if (p->kind != ORC_K_CSR) {
        double ca[8], cm[8], cn[8];
        orc_stencil_coeffs(p->kind, 0, p->h, p->beta, p->kappa, p->sigma, ca);
        orc_stencil_coeffs(p->kind, 1, p->h, p->beta, p->kappa, p->sigma, cm);
        orc_stencil_coeffs(p->kind, 2, p->h, p->beta, p->kappa, p->sigma, cn);
        g->A = make_stencil_op(p->kind, p->nx, p->ny, p->nz, ca);
        double ch[8], cs[8], cst[8];
        ch[0] = orc_round(prec, alpha + cm[0]);
        cs[0] = orc_round(prec, alpha);
        cst[0] = cs[0];
        for (int k = 1; k < 7; k++) {
            ch[k] = orc_round(prec, cm[k]);
            cs[k] = orc_round(prec, cn[k]);
            cst[k] = -cs[k];
        }
        ch[7] = 0.0;
        cs[7] = orc_round(prec, cn[7]);
        cst[7] = -cs[7];
        g->H = make_stencil_op(p->kind, p->nx, p->ny, p->nz, ch);
        g->S = make_stencil_op(p->kind, p->nx, p->ny, p->nz, cs);
        g->St = make_stencil_op(p->kind, p->nx, p->ny, p->nz, cst);
        fill_opf(&g->H, &g->Hf, NULL);
        fill_opf(&g->S, &g->Sf, NULL);
        fill_opf(&g->St, &g->Stf, NULL);
        if (p->kind == ORC_K_C2D5 && p->sigma_pt) {
            /* A carries T exactly; S and S^T carry +-T rounded to u_s */
            size_t np = (size_t)p->nx * p->ny;
            g->A.ep = p->sigma_pt;
            g->es_d = (double *)malloc(sizeof(double) * np);
            g->est_d = (double *)malloc(sizeof(double) * np);
            g->es_f = (float *)malloc(sizeof(float) * np);
            g->est_f = (float *)malloc(sizeof(float) * np);
            if (!g->es_d || !g->est_d || !g->es_f || !g->est_f) return -1;
            for (size_t i = 0; i < np; i++) {
                g->es_d[i] = orc_round(prec, p->sigma_pt[i]);
                g->est_d[i] = -g->es_d[i];
                g->es_f[i] = (float)g->es_d[i];
                g->est_f[i] = -g->es_f[i];
            }
            g->S.ep = g->es_d;
            g->St.ep = g->est_d;
            g->Sf.ep = g->es_f;
            g->Stf.ep = g->est_f;
        }
        return 0;
    }
    /* CSR: the pattern of M (= pattern of A + A^T) must hold every diagonal
     * entry; H, S and S^T are stored matrices on that pattern with the shift
     * added to the diagonal before rounding, as a precomputed H would be. */
    int n = p->n, nnzm = p->mrowptr[n];
    size_t nn = (size_t)(nnzm > 0 ? nnzm : 1);
    memset(&g->A, 0, sizeof g->A);
    g->A.kind = ORC_K_CSR; g->A.n = n; g->A.rowptr = p->rowptr; g->A.col = p->col;
    g->A.val = p->aval; g->A.d = 0.0;
    g->Mval_d = (double *)malloc(sizeof(double) * nn);
    g->Nval_d = (double *)malloc(sizeof(double) * nn);
    g->NvalT_d = (double *)malloc(sizeof(double) * nn);
    g->Mval_f = (float *)malloc(sizeof(float) * nn);
    g->Nval_f = (float *)malloc(sizeof(float) * nn);
    g->NvalT_f = (float *)malloc(sizeof(float) * nn);
    if (!g->Mval_d || !g->Nval_d || !g->NvalT_d || !g->Mval_f || !g->Nval_f || !g->NvalT_f)
        return -1;
    for (int i = 0; i < n; i++)
        for (int k = p->mrowptr[i]; k < p->mrowptr[i + 1]; k++) {
            double sh = (p->mcol[k] == i) ? alpha : 0.0;
            g->Mval_d[k] = orc_round(prec, p->mval[k] + sh);  /* H   */
            g->Nval_d[k] = orc_round(prec, p->nval[k] + sh);  /* S   */
            g->NvalT_d[k] = orc_round(prec, sh - p->nval[k]); /* S^T */
            g->Mval_f[k] = (float)g->Mval_d[k];
            g->Nval_f[k] = (float)g->Nval_d[k];
            g->NvalT_f[k] = (float)g->NvalT_d[k];
        }
    orc_op base;
    memset(&base, 0, sizeof base);
    base.kind = ORC_K_CSR; base.n = n; base.rowptr = p->mrowptr; base.col = p->mcol;
    base.d = 0.0;
    g->H = base; g->H.val = g->Mval_d;
    g->S = base; g->S.val = g->Nval_d;
    g->St = base; g->St.val = g->NvalT_d;
    fill_opf(&g->H, &g->Hf, g->Mval_f);
    fill_opf(&g->S, &g->Sf, g->Nval_f);
    fill_opf(&g->St, &g->Stf, g->NvalT_f);
    return 0;
}

static void free_ops(gadi_ops *g)
{
    free(g->Mval_d); free(g->Nval_d); free(g->NvalT_d);
    free(g->Mval_f); free(g->Nval_f); free(g->NvalT_f);
    free(g->es_d); free(g->est_d); free(g->es_f); free(g->est_f);
}

/* ------------------------------------------------------------------------ */
/* inner solvers                                                             */
/* ------------------------------------------------------------------------ */
/* Inner stopping rule (Sec. 5.1): relative residual of the inner system,
 * ||res_j|| <= tol ||res_0||, tested as res_j.res_j <= tol^2 res_0.res_0 in
 * double.  Early stop against stagnation (Sec. 5.1 names one without giving
 * it): stop when the residual has not reached a new minimum for `stag`
 * consecutive iterations (stag <= 0 disables it). */

static double dot_d(int m, const double *a, const double *b)
{
    double s = 0.0;
    OMP_FOR_SUM(s)
    for (int i = 0; i < m; i++) s = s + a[i] * b[i];
    return s;
}
/* FP32 dot product of stored FP32 vectors: the FP32 value nearest to the
 * exact dot product (products of floats are exact in double; the double sum
 * carries 29 more bits than the float result).  Order-independent, unlike
 * sequential FP32 accumulation, whose error grows with m. */
static float dot_f(int m, const float *a, const float *b)
{
    double s = 0.0;
    OMP_FOR_SUM(s)
    for (int i = 0; i < m; i++) s = s + (double)a[i] * (double)b[i];
    return (float)s;
}

/* CG on an SPD operator Op (H, or S^T S given as the pair S, St), double. */
static int cg_d(const orc_op *op1, const orc_op *op2, const double *rhs, double *xsol,
                double tol, int maxit, int stag, double *work)
{
    int m = op_len(op1);
    double *r = work, *p = work + m, *q = work + 2 * m, *u = work + 3 * m;
    memcpy(r, rhs, sizeof(double) * m);
    double rr = dot_d(m, r, r), rr0 = rr, best = rr, beta = 0.0;
    int since = 0, its = 0;
    for (int i = 0; i < m; i++) xsol[i] = 0.0;
    if (rr0 == 0.0) return 0;
    for (int j = 0; j < maxit; j++) {
        OMP_FOR
        for (int i = 0; i < m; i++) p[i] = (j == 0) ? r[i] : fma(beta, p[i], r[i]);
        double pq;
        if (op2 == NULL) {
            apply_d(op1, p, q);
            pq = dot_d(m, p, q);
        } else {
            apply_d(op1, p, u);          /* u = S p          */
            pq = dot_d(m, u, u);         /* p.S^T S p = u.u  */
            apply_d(op2, u, q);          /* q = S^T u        */
        }
        double a = rr / pq;
        OMP_FOR
        for (int i = 0; i < m; i++) {
            xsol[i] = (j == 0) ? a * p[i] : fma(a, p[i], xsol[i]);
            r[i] = fma(-a, q[i], r[i]);
        }
        double rn = dot_d(m, r, r);
        its = j + 1;
        if (rn <= tol * tol * rr0) break;
        if (!(rn == rn)) break;
        if (rn < best) { best = rn; since = 0; } else if (stag > 0 && ++since >= stag) break;
        beta = rn / rr;
        rr = rn;
    }
    return its;
}

/* The same in float arithmetic with u_s storage rounding. */
static int cg_f(const orc_op *op1, const op_f *f1, const orc_op *op2, const op_f *f2, int prec,
                const float *rhs, float *xsol, double tol, int maxit, int stag, float *work)
{
    int m = op_len(op1);
    float *r = work, *p = work + m, *q = work + 2 * m, *u = work + 3 * m;
    memcpy(r, rhs, sizeof(float) * m);
    float rr = dot_f(m, r, r), rr0 = rr, best = rr, beta = 0.0f;
    int since = 0, its = 0;
    for (int i = 0; i < m; i++) xsol[i] = 0.0f;
    if (rr0 == 0.0f) return 0;
    for (int j = 0; j < maxit; j++) {
        OMP_FOR
        for (int i = 0; i < m; i++) p[i] = st_f(prec, (j == 0) ? r[i] : r[i] + beta * p[i]);
        float pq;
        if (op2 == NULL) {
            apply_f(op1, f1, p, q);
            pq = dot_f(m, p, q);
        } else {
            apply_f(op1, f1, p, u);            /* u = S p, stored: rounded to u_s */
            OMP_FOR
            for (int i = 0; i < m; i++) u[i] = st_f(prec, u[i]);
            pq = dot_f(m, u, u);
            apply_f(op2, f2, u, q);
        }
        float a = rr / pq;
        OMP_FOR
        for (int i = 0; i < m; i++) {
            xsol[i] = st_f(prec, (j == 0) ? a * p[i] : xsol[i] + a * p[i]);
            r[i] = st_f(prec, r[i] - a * q[i]);
        }
        float rn = dot_f(m, r, r);
        its = j + 1;
        if ((double)rn <= tol * tol * (double)rr0) break;
        if (!(rn == rn)) break;
        if (rn < best) { best = rn; since = 0; } else if (stag > 0 && ++since >= stag) break;
        beta = rn / rr;
        rr = rn;
    }
    return its;
}

/* ------------------------------------------------------------------------ */
/* public single-step entry points (used by the per-step parity tests)       */
/* ------------------------------------------------------------------------ */
/* r_s in u_s (values as doubles) -> z in u_s: CG on H = alpha I + M. */
int orc_solve_h(const orc_problem *p, double alpha, int prec, const double *rs, double *z,
                double tol, int maxit, int stag)
{
    gadi_ops g;
    if (build_ops(p, alpha, prec, &g)) return -1;
    int m = op_len(&g.A), its;
    if (prec == ORC_FP64) {
        double *w = (double *)malloc(sizeof(double) * 4 * (size_t)(m > 0 ? m : 1));
        its = cg_d(&g.H, NULL, rs, z, tol, maxit, stag, w);
        free(w);
    } else {
        float *w = (float *)malloc(sizeof(float) * 6 * (size_t)(m > 0 ? m : 1));
        float *rf = w + 4 * m, *zf = w + 5 * m;
        OMP_FOR
        for (int i = 0; i < m; i++) rf[i] = (float)rs[i];
        its = cg_f(&g.H, &g.Hf, NULL, NULL, prec, rf, zf, tol, maxit, stag, w);
        OMP_FOR
        for (int i = 0; i < m; i++) z[i] = (double)zf[i];
        free(w);
    }
    free_ops(&g);
    return its;
}

/* z in u_s -> y in u_s: g = fl_s((2 - omega) alpha z), then CG on
 * S^T S y = S^T g (t0 = fl_s(S^T g)); or, with pointwise != 0 and the complex
 * problem, the exact diagonal solve y = fl_s(g / (alpha + i sigma)). */
int orc_solve_s(const orc_problem *p, double alpha, double omega, int prec, const double *z,
                double *y, double tol, int maxit, int stag, int pointwise)
{
    gadi_ops g;
    if (build_ops(p, alpha, prec, &g)) return -1;
    int m = op_len(&g.A), its = 0;
    double gam = (2.0 - omega) * alpha;
    if (prec == ORC_FP64) {
        double *w = (double *)malloc(sizeof(double) * 6 * (size_t)(m > 0 ? m : 1));
        double *gv = w + 4 * m, *t = w + 5 * m;
        for (int i = 0; i < m; i++) gv[i] = gam * z[i];
        if (pointwise && p->kind == ORC_K_C2D5) {
            for (int i = 0; i < m / 2; i++) {
                double ar = g.S.d, ai = g.S.ep ? g.S.ep[i] : g.S.e, den = ar * ar + ai * ai;
                double gr = gv[2 * i], gi = gv[2 * i + 1];
                y[2 * i] = (gr * ar + gi * ai) / den;
                y[2 * i + 1] = (gi * ar - gr * ai) / den;
            }
            its = 1;
        } else {
            apply_d(&g.St, gv, t);
            its = cg_d(&g.S, &g.St, t, y, tol, maxit, stag, w);
        }
        free(w);
    } else {
        float *w = (float *)malloc(sizeof(float) * 7 * (size_t)(m > 0 ? m : 1));
        float *gv = w + 4 * m, *t = w + 5 * m, *yf = w + 6 * m;
        float gamf = (float)gam;
        for (int i = 0; i < m; i++) gv[i] = st_f(prec, gamf * (float)z[i]);
        if (pointwise && p->kind == ORC_K_C2D5) {
            for (int i = 0; i < m / 2; i++) {
                float ar = g.Sf.d, ai = g.Sf.ep ? g.Sf.ep[i] : g.Sf.e, den = ar * ar + ai * ai;
                float gr = gv[2 * i], gi = gv[2 * i + 1];
                yf[2 * i] = st_f(prec, (gr * ar + gi * ai) / den);
                yf[2 * i + 1] = st_f(prec, (gi * ar - gr * ai) / den);
            }
            its = 1;
        } else {
            apply_f(&g.St, &g.Stf, gv, t);
            for (int i = 0; i < m; i++) t[i] = st_f(prec, t[i]);
            its = cg_f(&g.S, &g.Sf, &g.St, &g.Stf, prec, t, yf, tol, maxit, stag, w);
        }
        for (int i = 0; i < m; i++) y[i] = (double)yf[i];
        free(w);
    }
    free_ops(&g);
    return its;
}

/* One residual step (Algorithm 1, line "r = b - A x" in u_r = FP64, fused
 * with the previous update x = x + y in u = FP64):
 *   x_out = x + y (if y != NULL), r = b - A x_out, returns ||r||_2 and
 *   writes r_s = fl_s(r) (as doubles). */
double orc_residual(const orc_problem *p, int prec, const double *b, const double *x,
                    const double *y, double *x_out, double *r, double *rs)
{
    gadi_ops g;
    if (build_ops(p, 1.0, prec, &g)) return -1.0;
    int m = op_len(&g.A);
    double *ax = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    OMP_FOR
    for (int i = 0; i < m; i++) x_out[i] = y ? x[i] + y[i] : x[i];
    apply_d(&g.A, x_out, ax);
    double s = 0.0;
    OMP_FOR_SUM(s)
    for (int i = 0; i < m; i++) {
        r[i] = b[i] - ax[i];
        s = s + r[i] * r[i];
        rs[i] = orc_round(prec, r[i]);
    }
    free(ax);
    free_ops(&g);
    return sqrt(s);
}

/* ------------------------------------------------------------------------ */
/* residual in double-FP64 (u_r about u^2; Sec. 3.1 allows any u_r <= u)      */
/* ------------------------------------------------------------------------ */
/* Error-free transformations in double: a + b = s + e exactly (Knuth's
 * TwoSum), a * b = p + e exactly (the error by a fused multiply-add), as used
 * by the Dot2 algorithm of Ogita, Rump & Oishi, "Accurate sum and dot
 * product", SIAM J. Sci. Comput. 26(6), 2005. */
static void ef_sum(double a, double b, double *s, double *e)
{
    double ss = a + b;
    double bb = ss - a;
    *e = (a - (ss - bb)) + (b - bb);
    *s = ss;
}
static void ef_prod(double a, double b, double *p, double *e)
{
    double pp = a * b;
    *e = fma(a, b, -pp);
    *p = pp;
}
/* (hi, lo) -= a x: the product exact, its high part added by TwoSum, the two
 * error terms accumulated in lo */
static void dd_sub(double *hi, double *lo, double a, double x)
{
    double p, pe, q;
    ef_prod(-a, x, &p, &pe);
    ef_sum(*hi, p, hi, &q);
    *lo = *lo + (q + pe);
}

/* hi + lo rounded to u_s (|lo| at most half an ulp of hi).  For |hi| in the
 * normal binary32 range [2^-126, 2^128): to nearest among numbers with `sig`
 * significant bits (24 for FP32, 8 for BF16), a tie of hi decided by the sign
 * of lo (ties to even when lo = 0), overflow to infinity.  Elsewhere hi alone
 * is rounded.  FP64: hi. */
double orc_round_pair(int prec, double hi, double lo)
{
    if (prec == ORC_FP64) return hi;
    double a = fabs(hi);
    if (!(a >= ldexp(1.0, -126) && a < ldexp(1.0, 128))) return orc_round(prec, hi);
    int sig = prec == ORC_FP32 ? 24 : 8;
    double beyond = hi < 0 ? -lo : lo; /* > 0: the value lies past hi in magnitude */
    int e;
    (void)frexp(a, &e);                /* a in [2^(e-1), 2^e) */
    int q = e - sig;                   /* spacing of the target numbers there */
    double sc = ldexp(a, -q);          /* exact; in [2^(sig-1), 2^sig) */
    double fl = floor(sc), fr = sc - fl;
    double k;
    if (fr > 0.5) k = fl + 1.0;
    else if (fr < 0.5) k = fl;
    else if (beyond > 0) k = fl + 1.0;
    else if (beyond < 0) k = fl;
    else k = fmod(fl, 2.0) == 0.0 ? fl : fl + 1.0;
    double r = ldexp(k, q);
    if (r >= ldexp(1.0, 128)) r = INFINITY;
    return hi < 0 ? -r : r;
}

/* x_out = x + y (FP64); r = b - A x_out in double-FP64: per row b, then each
 * term of A's row in the operator's order (centre, W, E, S, N, B, T with zero
 * outside the grid, then the complex coupling; CSR: the stored row order),
 * renormalised by TwoSum into r_hi + r_lo; rs = the pair rounded to u_s.
 * Returns ||r_hi||_2. */
double orc_residual_dd(const orc_problem *p, int prec, const double *b, const double *x,
                       const double *y, double *x_out, double *r_hi, double *r_lo, double *rs)
{
    gadi_ops g;
    if (build_ops(p, 1.0, prec, &g)) return -1.0;
    const orc_op *A = &g.A;
    int m = op_len(A);
    for (int i = 0; i < m; i++) x_out[i] = y ? x[i] + y[i] : x[i];
    if (A->kind == ORC_K_CSR) {
        for (int i = 0; i < A->n; i++) {
            double hi = b[i], lo = 0.0;
            for (int k = A->rowptr[i]; k < A->rowptr[i + 1]; k++) dd_sub(&hi, &lo, A->val[k], x_out[A->col[k]]);
            ef_sum(hi, lo, &r_hi[i], &r_lo[i]);
        }
    } else {
        int nz = A->kind == ORC_K_3D7 ? A->nz : 1;
        int ndir = A->kind == ORC_K_3D7 ? 6 : 4;
        int cplx = A->kind == ORC_K_C2D5;
        int K = cplx ? 2 : 1;
        for (int iz = 0; iz < nz; iz++)
            for (int iy = 0; iy < A->ny; iy++)
                for (int ix = 0; ix < A->nx; ix++) {
                    long i = ((long)iz * A->ny + iy) * A->nx + ix;
                    for (int part = 0; part < K; part++) {
                        long ii = K * i + part;
                        double hi = b[ii], lo = 0.0;
                        dd_sub(&hi, &lo, A->d, x_out[ii]);
                        for (int dir = 0; dir < ndir; dir++) {
                            long j = nbr(A, ix, iy, iz, dir);
                            dd_sub(&hi, &lo, A->c[dir], j >= 0 ? x_out[K * j + part] : 0.0);
                        }
                        /* (i e) (xr + i xi) = -e xi + i e xr */
                        double ei = A->ep ? A->ep[i] : A->e;
                        if (cplx) dd_sub(&hi, &lo, part ? ei : -ei, x_out[K * i + (1 - part)]);
                        ef_sum(hi, lo, &r_hi[ii], &r_lo[ii]);
                    }
                }
    }
    double s = 0.0;
    for (int i = 0; i < m; i++) {
        s = s + r_hi[i] * r_hi[i];
        rs[i] = orc_round_pair(prec, r_hi[i], r_lo[i]);
    }
    free_ops(&g);
    return sqrt(s);
}

/* y = Op x in FP64 for the operator `which` (OP_A, OP_M, OP_N) of a problem. */
void orc_apply(const orc_problem *p, int which, const double *x, double *y)
{
    if (p->kind == ORC_K_CSR) {
        if (which == OP_A) orc_csr_apply(p->n, p->rowptr, p->col, p->aval, 0.0, x, y);
        else orc_csr_apply(p->n, p->mrowptr, p->mcol, which == OP_M ? p->mval : p->nval, 0.0, x, y);
        return;
    }
    double co[8];
    orc_stencil_coeffs(p->kind, which, p->h, p->beta, p->kappa, p->sigma, co);
    orc_op op = make_stencil_op(p->kind, p->nx, p->ny, p->nz, co);
    if (p->kind == ORC_K_C2D5 && p->sigma_pt && which != OP_M) op.ep = p->sigma_pt;
    apply_d(&op, x, y);
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1                                                               */
/* ------------------------------------------------------------------------ */
enum { ORC_OK = 0, ORC_NOT_CONVERGED = 1, ORC_STAGNATED = 2, ORC_DIVERGED = 3 };

typedef struct {
    double tol_h, tol_s;
    int maxit_inner, inner_stag, outer_stag_window, s_pointwise;
    int ur_dd; /* 1: the residual in double-FP64 (orc_residual_dd) */
} orc_opts;

typedef struct {
    int outer_its;
    long inner_h, inner_s;
    double relres;
    int status;
} orc_stats;

/* x (in/out): initial guess in, last iterate out.  hist (nullable) receives
 * relres_k = ||b - A x_k|| / ||b - A x_0|| for k = 0 .. outer_its. */
int orc_gadi(const orc_problem *p, const double *b, double *x, double alpha, double omega,
             int prec, double tol, int maxit, const orc_opts *o, orc_stats *st, double *hist)
{
    gadi_ops g;
    if (build_ops(p, alpha, prec, &g)) return -1;
    int m = op_len(&g.A);
    size_t mm = (size_t)(m > 0 ? m : 1);
    double *xn = (double *)malloc(sizeof(double) * mm), *r = (double *)malloc(sizeof(double) * mm);
    double *rs = (double *)malloc(sizeof(double) * mm), *z = (double *)malloc(sizeof(double) * mm);
    double *y = (double *)malloc(sizeof(double) * mm);
    double *rl = (double *)malloc(sizeof(double) * mm);
    memset(st, 0, sizeof *st);
    double r0 = -1.0;
    int status = ORC_NOT_CONVERGED, k;
    for (k = 0;; k++) {
        double rn = o->ur_dd ? orc_residual_dd(p, prec, b, x, k > 0 ? y : NULL, xn, r, rl, rs)
                             : orc_residual(p, prec, b, x, k > 0 ? y : NULL, xn, r, rs);
        memcpy(x, xn, sizeof(double) * m);
        if (k == 0) r0 = rn;
        /* r0 = 0: x_0 solves the system; a non-finite r0 gives a NaN relres */
        double rel = (r0 == 0.0) ? 0.0 : rn / r0;
        if (hist) hist[k] = rel;
        st->relres = rel;
        if (rel <= tol) { status = ORC_OK; break; }
        if (!(rel == rel) || isinf(rel) || rel > 1e6) { status = ORC_DIVERGED; break; }
        if (o->outer_stag_window > 0 && hist && k >= o->outer_stag_window &&
            rel > 0.99 * hist[k - o->outer_stag_window]) { status = ORC_STAGNATED; break; }
        if (k >= maxit) { status = ORC_NOT_CONVERGED; break; }
        st->inner_h += orc_solve_h(p, alpha, prec, rs, z, o->tol_h, o->maxit_inner, o->inner_stag);
        st->inner_s += orc_solve_s(p, alpha, omega, prec, z, y, o->tol_s, o->maxit_inner,
                                   o->inner_stag, o->s_pointwise);
    }
    st->outer_its = k;
    st->status = status;
    free(xn); free(r); free(rs); free(z); free(y); free(rl);
    free_ops(&g);
    return status;
}
