/* Assembled-CSR FP64 Jacobi-PCG and the element steps of one OC iteration,
 * plain C with OpenMP, for timing the oracle on the host's cores.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by bench.py's CPU baseline (and the tests
 * that check it); the CUDA library never links or calls it and they share no
 * code.  Built by oracle/build_c.py with gcc -O2 -fopenmp.
 *
 * What it computes follows the paper's statement of the method:
 *   - K = sum_e E_e P_e^T KE P_e assembled as CSR (Section 2.2: element
 *     matrices scattered into the global sparse matrix), clamped dofs made
 *     identity rows and columns (Section 2.2, "modifying the system matrix");
 *     KE is passed in (the NumPy oracle's Gauss-quadrature element);
 *   - the solve K u = f by Jacobi-preconditioned CG to ||f - K u|| <= rtol ||f||
 *     (the paper uses a direct solver; iterative here, as on the GPU);
 *   - element energies ce_e = u_e^T KE u_e, sensitivities
 *     dc_e = -p x_e^(p-1) (E0 - Emin) ce_e (Section 2.3);
 *   - the sensitivity filter with weights max(0, rmin - distance) between
 *     element centroids, normalised by the in-grid row sums (Section 2.4);
 *   - OC bisection on the volume multiplier (Section 2.3).
 * Node (i,j,k) = i + nx (j + ny k), dof 3 node + c, element
 * e = i + nelx (j + nely k), local node a + 2b + 4c at corner (a,b,c). */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int64_t n;          /* rows */
    int64_t* rowptr;    /* [n + 1] */
    int32_t* col;       /* [nnz] */
    double* val;        /* [nnz] */
} csr_t;

static void elem_dofs(int nelx, int nely, int i, int j, int k, int64_t* ed) {
    const int64_t nx = nelx + 1, ny = nely + 1;
    for (int c = 0; c < 2; ++c)
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) {
                const int64_t node = (i + a) + nx * ((j + b) + ny * (int64_t)(k + c));
                const int loc = a + 2 * b + 4 * c;
                for (int d = 0; d < 3; ++d) ed[3 * loc + d] = 3 * node + d;
            }
}

int omp_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Build the clamped CSR operator.  Every row of a structured hex grid has its
 * columns at the 27 neighbouring nodes (3 dofs each): the pattern is laid out
 * first, then each element adds E_e KE into it (rows owned by the thread that
 * owns the element's first node plane are not shared, so the scatter uses
 * atomics).  Returns 0 on success. */
int csr_assemble(int nelx, int nely, int nelz, const double* E, const double* KE,
                 const uint8_t* fixed, csr_t* K) {
    const int64_t nx = nelx + 1, ny = nely + 1, nz = nelz + 1;
    const int64_t N = nx * ny * nz, n = 3 * N;
    K->n = n;
    K->rowptr = (int64_t*)malloc(sizeof(int64_t) * (n + 1));
    if (!K->rowptr) return 1;
    K->rowptr[0] = 0;
    for (int64_t node = 0; node < N; ++node) {
        const int64_t i = node % nx, j = (node / nx) % ny, k = node / (nx * ny);
        int64_t cnt = 0;
        for (int dk = -1; dk <= 1; ++dk)
            for (int dj = -1; dj <= 1; ++dj)
                for (int di = -1; di <= 1; ++di)
                    if (i + di >= 0 && i + di < nx && j + dj >= 0 && j + dj < ny && k + dk >= 0 &&
                        k + dk < nz)
                        cnt += 3;
        for (int d = 0; d < 3; ++d) K->rowptr[3 * node + d + 1] = K->rowptr[3 * node + d] + cnt;
    }
    const int64_t nnz = K->rowptr[n];
    K->col = (int32_t*)malloc(sizeof(int32_t) * nnz);
    K->val = (double*)calloc((size_t)nnz, sizeof(double));
    if (!K->col || !K->val) return 1;
#pragma omp parallel for schedule(static)
    for (int64_t node = 0; node < N; ++node) {
        const int64_t i = node % nx, j = (node / nx) % ny, k = node / (nx * ny);
        for (int d = 0; d < 3; ++d) {
            int64_t p = K->rowptr[3 * node + d];
            for (int dk = -1; dk <= 1; ++dk)
                for (int dj = -1; dj <= 1; ++dj)
                    for (int di = -1; di <= 1; ++di)
                        if (i + di >= 0 && i + di < nx && j + dj >= 0 && j + dj < ny && k + dk >= 0 &&
                            k + dk < nz) {
                            const int64_t m = (i + di) + nx * ((j + dj) + ny * (k + dk));
                            for (int e = 0; e < 3; ++e) K->col[p++] = (int32_t)(3 * m + e);
                        }
        }
    }
    const int64_t nel = (int64_t)nelx * nely * nelz;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < nel; ++e) {
        const int i = (int)(e % nelx), j = (int)((e / nelx) % nely), k = (int)(e / ((int64_t)nelx * nely));
        int64_t ed[24];
        elem_dofs(nelx, nely, i, j, k, ed);
        for (int a = 0; a < 24; ++a) {
            const int64_t row = ed[a];
            const int64_t r0 = K->rowptr[row], r1 = K->rowptr[row + 1];
            for (int b = 0; b < 24; ++b) {
                const int32_t cidx = (int32_t)ed[b];
                /* columns of a row are sorted: binary search */
                int64_t lo = r0, hi = r1 - 1;
                while (lo < hi) {
                    const int64_t mid = (lo + hi) / 2;
                    if (K->col[mid] < cidx) lo = mid + 1;
                    else hi = mid;
                }
                const double v = E[e] * KE[a * 24 + b];
#pragma omp atomic
                K->val[lo] += v;
            }
        }
    }
    /* clamped dofs: identity rows and columns */
#pragma omp parallel for schedule(static)
    for (int64_t row = 0; row < n; ++row)
        for (int64_t p = K->rowptr[row]; p < K->rowptr[row + 1]; ++p) {
            const int64_t cidx = K->col[p];
            if (fixed[row] || fixed[cidx]) K->val[p] = (row == cidx) ? 1.0 : 0.0;
        }
    return 0;
}

void csr_free(csr_t* K) {
    free(K->rowptr);
    free(K->col);
    free(K->val);
    K->rowptr = NULL;
    K->col = NULL;
    K->val = NULL;
}

static void spmv(const csr_t* K, const double* x, double* y) {
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < K->n; ++r) {
        double s = 0.0;
        for (int64_t p = K->rowptr[r]; p < K->rowptr[r + 1]; ++p) s += K->val[p] * x[K->col[p]];
        y[r] = s;
    }
}

static double dot(int64_t n, const double* a, const double* b) {
    double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* Jacobi-PCG from u (in/out) for at most maxit iterations or until the
 * recurrence residual is <= rtol |f|; returns the iterations done. */
int64_t csr_jacobi_pcg(const csr_t* K, const double* f, double* u, double rtol, int64_t maxit) {
    const int64_t n = K->n;
    double *r = malloc(sizeof(double) * n), *z = malloc(sizeof(double) * n),
           *p = malloc(sizeof(double) * n), *q = malloc(sizeof(double) * n),
           *dinv = malloc(sizeof(double) * n);
    if (!r || !z || !p || !q || !dinv) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t row = 0; row < n; ++row) {
        double d = 1.0;
        for (int64_t k = K->rowptr[row]; k < K->rowptr[row + 1]; ++k)
            if (K->col[k] == row) d = K->val[k];
        dinv[row] = 1.0 / d;
    }
    spmv(K, u, q);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        r[i] = f[i] - q[i];
        z[i] = dinv[i] * r[i];
        p[i] = z[i];
    }
    const double fn = sqrt(dot(n, f, f));
    double rz = dot(n, r, z);
    int64_t it = 0;
    while (it < maxit && sqrt(dot(n, r, r)) > rtol * fn) {
        spmv(K, p, q);
        const double alpha = rz / dot(n, p, q);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            u[i] += alpha * p[i];
            r[i] -= alpha * q[i];
            z[i] = dinv[i] * r[i];
        }
        const double rzn = dot(n, r, z);
        const double beta = rzn / rz;
        rz = rzn;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
        ++it;
    }
    free(r);
    free(z);
    free(p);
    free(q);
    free(dinv);
    return it;
}

/* ce_e = u_e^T KE u_e, dc_e = -p x^(p-1) (E0 - Emin) ce_e; returns the
 * compliance sum_e E_e ce_e. */
double element_steps(int nelx, int nely, int nelz, const double* KE, const double* u, const double* x,
                     double penal, double E0, double Emin, double* ce, double* dc) {
    const int64_t nel = (int64_t)nelx * nely * nelz;
    double comp = 0.0;
#pragma omp parallel for reduction(+ : comp) schedule(static)
    for (int64_t e = 0; e < nel; ++e) {
        const int i = (int)(e % nelx), j = (int)((e / nelx) % nely), k = (int)(e / ((int64_t)nelx * nely));
        int64_t ed[24];
        elem_dofs(nelx, nely, i, j, k, ed);
        double s = 0.0;
        for (int a = 0; a < 24; ++a) {
            double t = 0.0;
            for (int b = 0; b < 24; ++b) t += KE[a * 24 + b] * u[ed[b]];
            s += u[ed[a]] * t;
        }
        ce[e] = s;
        const double xe = x[e];
        comp += (Emin + pow(xe, penal) * (E0 - Emin)) * s;
        dc[e] = -penal * pow(xe, penal - 1.0) * (E0 - Emin) * s;
    }
    return comp;
}

/* dcf_e = sum_i H_ei x_i dc_i / (Hs_e max(1e-3, x_e)), H_ei = max(0, rmin - |c_e - c_i|) */
void sensitivity_filter(int nelx, int nely, int nelz, double rmin, const double* x, const double* dc,
                        double* dcf) {
    const int R = (int)ceil(rmin) - 1;
    const int64_t nel = (int64_t)nelx * nely * nelz;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < nel; ++e) {
        const int i = (int)(e % nelx), j = (int)((e / nelx) % nely), k = (int)(e / ((int64_t)nelx * nely));
        double num = 0.0, hs = 0.0;
        for (int dk = -R; dk <= R; ++dk)
            for (int dj = -R; dj <= R; ++dj)
                for (int di = -R; di <= R; ++di) {
                    const int ii = i + di, jj = j + dj, kk = k + dk;
                    if (ii < 0 || ii >= nelx || jj < 0 || jj >= nely || kk < 0 || kk >= nelz) continue;
                    const double w = rmin - sqrt((double)(di * di + dj * dj + dk * dk));
                    if (w <= 0.0) continue;
                    const int64_t m = ii + (int64_t)nelx * (jj + (int64_t)nely * kk);
                    num += w * x[m] * dc[m];
                    hs += w;
                }
        dcf[e] = num / (hs * fmax(1e-3, x[e]));
    }
}

/* OC bisection: x_new = clamp(x sqrt(-dcf / lambda), max(0, x - move),
 * min(1, x + move)) on design elements (passive pinned: 1 void -> 0, 2
 * solid -> 1); lambda in [0, 1e9] until (l2 - l1) / (l1 + l2) <= tol, the
 * design volume above volfrac * n_design raising l1.  Returns halvings. */
int oc_update(int64_t nel, const double* x, const double* dcf, const uint8_t* passive, double volfrac,
              double move, double tol, double* xnew) {
    int64_t ndes = 0;
    for (int64_t e = 0; e < nel; ++e) ndes += passive ? (passive[e] == 0) : 1;
    const double target = volfrac * (double)ndes;
    double l1 = 0.0, l2 = 1e9;
    int h = 0;
    while ((l2 - l1) / (l1 + l2) > tol && h < 400) {
        const double lmid = 0.5 * (l1 + l2);
        double vol = 0.0;
#pragma omp parallel for reduction(+ : vol) schedule(static)
        for (int64_t e = 0; e < nel; ++e) {
            const uint8_t t = passive ? passive[e] : 0;
            double v;
            if (t == 1) v = 0.0;
            else if (t == 2) v = 1.0;
            else {
                const double b = x[e] * sqrt(fmax(0.0, -dcf[e]) / lmid);
                v = fmax(0.0, fmax(x[e] - move, fmin(1.0, fmin(x[e] + move, b))));
                vol += v;
            }
            xnew[e] = v;
        }
        if (vol > target) l1 = lmid;
        else l2 = lmid;
        ++h;
    }
    return h;
}
