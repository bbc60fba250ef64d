// Kernel parameter block shared by the host driver and the device code.
#pragma once
#include <cstddef>
#include <cstdint>

namespace gadi {

// threads per block of the persistent kernels (host and device agree on it):
// one block of 512 threads per SM -- the grid barrier and the grid-wide sums
// then involve one block per SM, which measured faster than two blocks of
// 256 at the same thread count
#ifndef GADI_THREADS
#define GADI_THREADS 512
#endif

enum : int { P_FP64 = 0, P_FP32 = 1, P_BF16 = 2 };
enum : int { K_2D5 = 0, K_3D7 = 1, K_C2D5 = 2, K_CSR = 3 };

enum : int {
    MODE_SOLVE = 0,    // Algorithm 1, all outer iterations
    MODE_RESIDUAL = 1, // one residual step
    MODE_SOLVE_H = 2,  // one H-solve (CG)
    MODE_SOLVE_S = 3,  // one S-solve (CGNR or pointwise)
    MODE_APPLY = 4     // y = Op x in FP64
};

// A 7-point coefficient set: centre d, neighbours c (W, E, S, N, B, T) and
// the complex class's imaginary diagonal e.
template <class C> struct Coef7 {
    C d, c[6], e;
};

// Device-written results of a launch.
struct Ctl {
    int status;
    int outer_its;
    long long inner_h, inner_s;
    double relres, r0, rnorm;
    int x_in_x1;   // 1 if the final iterate sits in the x1 work buffer
    int pad;
};

// Operator coefficients.  A is FP64.  H, S and S^T hold values already rounded
// to u_s on the host (exactly representable in the compute type).
struct Coefs {
    double a_d, a_c[6], a_e;
    double h_d, h_c[6];
    double s_d, s_c[6], s_e;
    double t_d, t_c[6], t_e; // S^T (S^H for the complex class)
    double gamma;            // (2 - omega) alpha, rounded to the compute type
    double m_d, m_c[6];      // M in FP64 (for gadi_apply)
    double n_c[6], n_e;      // N in FP64 (for gadi_apply)
};

struct Params {
    int kind, prec, mode, op; // op: gadi_op for MODE_APPLY
    int nx, ny, nz;
    long long npts, nelem; // nelem = doubles per outer vector
    Coefs co;
    // H, S, S^T of `co` as sets in FP32 (the FP32/BF16 compute type) and
    // FP64 (H's e = 0); filled from `co` by fill_coef_sets before launch
    Coef7<float> hf, sf, tf;
    Coef7<double> hd, sd, td;
    // k if A's centre coefficient co.a_d is 2^k (|k| < 1000), else kNoPow2:
    // the residual then forms a_d x by adding k to x's exponent
    int ad_pow2;
    // CSR (device arrays)
    const int *rowptr, *col;
    const double *aval;                 // A
    const int *mrowptr, *mcol;          // pattern of M (with full diagonal)
    const double *mval_d, *nval_d;      // M, N in FP64
    const void *hval, *sval, *tval;     // H, S, S^T in u_s on M's pattern
    // vectors
    const double *b;
    double *x, *x1, *r_out;
    double *r_lo_out;  // double-FP64 residual: the low part (nullable)
    void *r, *z, *p0, *p1, *y, *u; // u_s storage
    void *q;                       // compute type (CSR only)
    const double *ax_in;           // MODE_APPLY input
    double *ax_out;                // MODE_APPLY output
    // control
    double tol, tol_h, tol_s;
    int maxit, maxit_inner, inner_stag, outer_win, pointwise, first_y_null;
    int resident;  // 1: the H-solve keeps p in shared memory (2D, FP32/BF16);
                   // 2: also z and r in tensor memory
    int s_resident; // with resident = 2 in MODE_SOLVE: CGNR on S with p in
                    // shared memory and t, y in tensor memory (blocks of >= 2 rows)
    int ur_dd;     // 1: the residual in double-FP64 (u_r ~ u^2)
    // complex class with a per-point imaginary diagonal T = diag(sig) (FP64,
    // one value per grid point; null: the scalar sigma of the coefficients);
    // sig_a: the sign T carries in the FP64 set `a` (A, N: +1, A^T: -1, M: 0)
    const double *sig;
    double sig_a;
    // a batched unit of four interleaved right-hand sides: the iterate (two
    // ping-pong buffers) and the right-hand sides as [n][4] FP64 work
    // vectors; x and b above are then the caller's [4][n] arrays
    double *xm0, *xm1, *bm;
    double *part;  // 2 slots x 2 values x gridDim doubles
    double *hist;  // maxit + 1 doubles (device)
    Ctl *ctl;
    unsigned long long *bar;
    int *abort_flag;
};

constexpr int kNoPow2 = 1 << 30;

// Derive the coefficient sets hf/sf/tf and hd/sd/td and ad_pow2 from P.co
// (host side, before every launch; FP32 by round to nearest, as a device
// conversion).
inline void fill_coef_sets(Params &P)
{
    const Coefs &c = P.co;
    P.ad_pow2 = kNoPow2;
    {
        uint64_t u;
        static_assert(sizeof(double) == sizeof(uint64_t), "binary64");
        __builtin_memcpy(&u, &c.a_d, 8);
        const int ex = (int)((u >> 52) & 0x7ff);
        // a positive normal power of two: sign 0, fraction 0
        if ((u >> 63) == 0 && (u & 0xfffffffffffffull) == 0 && ex != 0 && ex != 0x7ff) P.ad_pow2 = ex - 1023;
    }
    P.hd.d = c.h_d; P.hd.e = 0.0;
    P.sd.d = c.s_d; P.sd.e = c.s_e;
    P.td.d = c.t_d; P.td.e = c.t_e;
    for (int k = 0; k < 6; k++) {
        P.hd.c[k] = c.h_c[k];
        P.sd.c[k] = c.s_c[k];
        P.td.c[k] = c.t_c[k];
    }
    const Coef7<double> *d[3] = {&P.hd, &P.sd, &P.td};
    Coef7<float> *f[3] = {&P.hf, &P.sf, &P.tf};
    for (int i = 0; i < 3; i++) {
        f[i]->d = (float)d[i]->d;
        f[i]->e = (float)d[i]->e;
        for (int k = 0; k < 6; k++) f[i]->c[k] = (float)d[i]->c[k];
    }
}

// One batched launch: units (system, right-hand side) taken from queues by
// groups of blocks.  Groups are contiguous block ranges of sizes chosen per
// size class of the units (the host's tuner); group g owns blocks
// [group_first[g], group_first[g] + group_size[g]) and takes units of its
// class first, then of the other classes (largest first) once its own queue
// is empty.  Per-group state is strided by group index.
struct BatchParams {
    Params *units;   // device array, one per unit; the group leader patches the work pointers
    int nunits;
    int ngroups, nclasses;
    const int *block_group;  // per block: its group
    const int *group_first;  // per group: first block
    const int *group_size;   // per group: blocks
    const int *group_class;  // per group: its size class
    const int *class_begin;  // per class c: its units are order[class_begin[c] .. class_begin[c+1])
    const int *class_gmin;   // per class: the group sizes that may take its units are
    const int *class_gmax;   // [class_gmin, class_gmax] (the resident H-solve's limits)
    const int *order;        // unit indices by class, largest system first within a class
    int *queue;      // per class (stride 32 ints): units taken so far (zeroed before launch)
    int *group_unit; // per group (stride 32 ints): the unit it is working on
    // per-group work: x1 (FP64) and six u_s vectors, each slab_bytes long
    char *work;
    size_t group_work_bytes, slab_bytes, slab_d_bytes;
    double *part;   // 4 doubles per block, a group's slots start at 4 * group_first
    unsigned long long *bar; // per group barrier counter (stride 8)
    double *hist;   // per group hist_len doubles
    int hist_len;
    Ctl *ctl;       // per unit
    unsigned long long *t0, *t1; // per unit start / end (globaltimer ns)
    int *abort_flag;
};
} // namespace gadi
