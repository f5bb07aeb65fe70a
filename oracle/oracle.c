/*
 * Plain CPU oracle for the triangular-domain maps and their workloads.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path includes,
 * links or calls this file; only the tests, the smoke check and the bench's
 * CPU-baseline leg do.  It shares no code with the CUDA sources.
 *
 * Everything here is the slow, obvious form of what the paper defines:
 * nested loops in the order the definitions are written, FP64 wherever
 * floating point is involved, no blocking or algebraic rewriting.  OpenMP
 * only splits independent outer-loop iterations across host threads; every
 * floating-point sum keeps a fixed order that does not depend on the thread
 * count.
 *
 * Paper: C. A. Navarro, B. Bustos, N. Hitschfeld, "A Non-linear GPU Thread
 * Map for Triangular Domains" (arXiv 1609.01490).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------
 * Section 3.1, Eq. (eq_matrix_indexing): the blocks of the lower triangle
 * are numbered row by row, left to right.  Walking that matrix with a running
 * counter gives the map omega -> (i, j) by enumeration, with no square root.
 * with_diag = 0 enumerates the strict triangle j < i (the variant of
 * Eq. eq_theorem_nodiag).  Returns the number of entries written.
 * ------------------------------------------------------------------------ */
int64_t orc_lambda_enum(int64_t m, int with_diag, uint32_t *oi, uint32_t *oj)
{
    int64_t w = 0;
    for (int64_t i = 0; i < m; ++i) {
        int64_t jend = with_diag ? i + 1 : i;
        for (int64_t j = 0; j < jend; ++j) {
            oi[w] = (uint32_t)i;
            oj[w] = (uint32_t)j;
            ++w;
        }
    }
    return w;
}

/* ------------------------------------------------------------------------
 * Section 6: blocks of the discrete tetrahedron, numbered layer by layer,
 * each layer a triangle numbered as in Eq. (eq_matrix_indexing).  Block omega
 * -> (layer, row, col) with layer >= row >= col.
 * ------------------------------------------------------------------------ */
int64_t orc_tet_enum(int64_t m, uint32_t *ol, uint32_t *orow, uint32_t *ocol)
{
    int64_t w = 0;
    for (int64_t l = 0; l < m; ++l)
        for (int64_t r = 0; r <= l; ++r)
            for (int64_t c = 0; c <= r; ++c) {
                ol[w] = (uint32_t)l;
                orow[w] = (uint32_t)r;
                ocol[w] = (uint32_t)c;
                ++w;
            }
    return w;
}

/* ------------------------------------------------------------------------
 * Section 5, test 2 (and the commented definition beside it): the Euclidean
 * distance of every pair i >= j,
 *     d_ij = sqrt( sum_k (x_ik - x_jk)^2 ),
 * evaluated in FP64 from the FP32 inputs and stored row-major into the packed
 * lower triangle with diagonal, entry i(i+1)/2 + j (Eq. eq_matrix_indexing
 * applied to elements).  Rows [r0, r1) only; out[0] holds pair (r0, 0).
 * ------------------------------------------------------------------------ */
void orc_edm_rows(const float *x, int64_t n, int64_t d, int64_t r0, int64_t r1, double *out)
{
    (void)n;
    const int64_t base = r0 * (r0 + 1) / 2;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = r0; i < r1; ++i) {
        double *row = out + (i * (i + 1) / 2 - base);
        for (int64_t j = 0; j <= i; ++j) {
            double s = 0.0;
            for (int64_t k = 0; k < d; ++k) {
                double diff = (double)x[i * d + k] - (double)x[j * d + k];
                s += diff * diff;
            }
            row[j] = sqrt(s);
        }
    }
}

/* The same distance for an explicit list of pairs (used to check samples of
 * outputs too large to recompute whole). */
void orc_edm_pairs(const float *x, int64_t d, const int64_t *pi, const int64_t *pj,
                   int64_t npairs, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < npairs; ++p) {
        double s = 0.0;
        for (int64_t k = 0; k < d; ++k) {
            double diff = (double)x[pi[p] * d + k] - (double)x[pj[p] * d + k];
            s += diff * diff;
        }
        out[p] = sqrt(s);
    }
}

/* ------------------------------------------------------------------------
 * Cellular automaton on the triangular domain (Section 1 lists the cellular
 * automaton on a triangle among the TD problems).  One synchronous step of
 * an outer-totalistic rule over the Moore neighbourhood: a cell is alive when
 * its byte is non-zero; it is alive next step when
 *     alive  and bit count of survive_mask is set, or
 *     dead   and bit count of birth_mask is set,
 * where count is the number of alive neighbours among the 8 around it.  The
 * domain is {(i, j): 0 <= j <= i < n}; every position outside it counts as
 * dead.  Only domain cells of `out` are written (as 0 or 1); the rest of
 * `out` is left as it was.
 * ------------------------------------------------------------------------ */
static int orc_alive(const uint8_t *g, int64_t n, int64_t ld, int64_t i, int64_t j)
{
    if (i < 0 || j < 0 || i >= n || j > i)
        return 0;
    return g[i * ld + j] != 0;
}

void orc_ca_step(const uint8_t *in, uint8_t *out, int64_t n, int64_t ld,
                 uint32_t birth_mask, uint32_t survive_mask)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = 0; j <= i; ++j) {
            int count = 0;
            for (int di = -1; di <= 1; ++di)
                for (int dj = -1; dj <= 1; ++dj)
                    if (di != 0 || dj != 0)
                        count += orc_alive(in, n, ld, i + di, j + dj);
            int alive = orc_alive(in, n, ld, i, j);
            uint32_t mask = alive ? survive_mask : birth_mask;
            out[i * ld + j] = (uint8_t)((mask >> count) & 1u);
        }
    }
}

/* `steps` synchronous steps, alternating between two buffers; the result is
 * left in `a` when steps is even and in `b` when it is odd. */
void orc_ca_run(uint8_t *a, uint8_t *b, int64_t n, int64_t ld, uint32_t birth_mask,
                uint32_t survive_mask, int64_t steps)
{
    for (int64_t s = 0; s < steps; ++s) {
        if (s % 2 == 0)
            orc_ca_step(a, b, n, ld, birth_mask, survive_mask);
        else
            orc_ca_step(b, a, n, ld, birth_mask, survive_mask);
    }
}

/* ------------------------------------------------------------------------
 * Triplet interaction on the tetrahedral domain (Section 6 names
 * triplet-interaction n-body problems).  The Axilrod-Teller triple-dipole
 * energy of N points,
 *     E = sum_{i>j>k} nu (1 + 3 cos g_i cos g_j cos g_k) / (r_ij r_jk r_ki)^3,
 * with g_v the interior angle of triangle (i, j, k) at vertex v, taken from
 * the dot product of the two edge vectors leaving v.  FP64 throughout.  Each
 * i sums its (j, k) terms in a fixed order; the per-i sums are then added in
 * increasing i with Kahan compensation, so the result does not depend on the
 * thread count.  abs_sum receives sum |term| (the scale for error bounds).
 * ------------------------------------------------------------------------ */
static double orc_at_term(const float *p, int64_t i, int64_t j, int64_t k, double nu)
{
    const float *a = p + 3 * i, *b = p + 3 * j, *c = p + 3 * k;
    double ab[3], ac[3], bc[3];
    for (int t = 0; t < 3; ++t) {
        ab[t] = (double)b[t] - (double)a[t];
        ac[t] = (double)c[t] - (double)a[t];
        bc[t] = (double)c[t] - (double)b[t];
    }
    double lab = sqrt(ab[0] * ab[0] + ab[1] * ab[1] + ab[2] * ab[2]);
    double lac = sqrt(ac[0] * ac[0] + ac[1] * ac[1] + ac[2] * ac[2]);
    double lbc = sqrt(bc[0] * bc[0] + bc[1] * bc[1] + bc[2] * bc[2]);
    /* angle at a between a->b and a->c; at b between b->a and b->c; at c
     * between c->a and c->b */
    double cos_a = (ab[0] * ac[0] + ab[1] * ac[1] + ab[2] * ac[2]) / (lab * lac);
    double cos_b = (-ab[0] * bc[0] - ab[1] * bc[1] - ab[2] * bc[2]) / (lab * lbc);
    double cos_c = (ac[0] * bc[0] + ac[1] * bc[1] + ac[2] * bc[2]) / (lac * lbc);
    double prod = lab * lbc * lac;
    return nu * (1.0 + 3.0 * cos_a * cos_b * cos_c) / (prod * prod * prod);
}

double orc_at_energy(const float *p, int64_t n, double nu, double *abs_sum)
{
    double *part = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *apart = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0, sa = 0.0;
        for (int64_t j = 0; j < i; ++j)
            for (int64_t k = 0; k < j; ++k) {
                double t = orc_at_term(p, i, j, k, nu);
                s += t;
                sa += fabs(t);
            }
        part[i] = s;
        apart[i] = sa;
    }
    double e = 0.0, comp = 0.0, ea = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double y = part[i] - comp;
        double t = e + y;
        comp = (t - e) - y;
        e = t;
        ea += apart[i];
    }
    free(part);
    free(apart);
    if (abs_sum)
        *abs_sum = ea;
    return e;
}

/* The same energy over the triplets of a range of tetrahedral blocks only:
 * the triplet i > j > k lies in block (L, R, C) = (i / rho, j / rho, k / rho),
 * L >= R >= C, whose number in the order of orc_tet_enum (layer L, then row
 * R <= L, then column C <= R; Section 6) is the count of blocks before it,
 *     w = L(L+1)(L+2)/6 + R(R+1)/2 + C,
 * and the triplet counts when w0 <= w < w1.  The terms of one i are added in
 * the order of orc_at_energy, so the whole range [0, T_m) gives its result
 * bit for bit. */
double orc_at_energy_blocks(const float *p, int64_t n, double nu, int64_t rho, int64_t w0, int64_t w1,
                            double *abs_sum)
{
    double *part = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *apart = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0, sa = 0.0;
        const int64_t L = i / rho;
        for (int64_t j = 0; j < i; ++j) {
            const int64_t R = j / rho;
            for (int64_t k = 0; k < j; ++k) {
                const int64_t C = k / rho;
                const int64_t w = L * (L + 1) * (L + 2) / 6 + R * (R + 1) / 2 + C;
                if (w < w0 || w >= w1)
                    continue;
                double t = orc_at_term(p, i, j, k, nu);
                s += t;
                sa += fabs(t);
            }
        }
        part[i] = s;
        apart[i] = sa;
    }
    double e = 0.0, comp = 0.0, ea = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double y = part[i] - comp;
        double t = e + y;
        comp = (t - e) - y;
        e = t;
        ea += apart[i];
    }
    free(part);
    free(apart);
    if (abs_sum)
        *abs_sum = ea;
    return e;
}

/* ------------------------------------------------------------------------
 * Section 5, test 3: collision detection of N spheres with random radii.
 * Spheres i and j (i > j) collide when the distance between their centres is
 * at most r_i + r_j (touching counts), tested on squares so that no root is
 * taken:
 *     s = sum_k (c_i,k - c_j,k)^2  (k = 0 .. dim-1, added in increasing k),
 *     collide  <=>  s <= (r_i + r_j)^2.
 * The paper fixes no precision.  Because this floating-point test decides an
 * integer result, it is taken here in FP32, the precision of the GPU path:
 * every difference, square, sum and the comparison are single IEEE FP32
 * operations rounded to nearest, in the order written above (the build
 * turns contraction into fused multiply-adds off).  Centres are row-major
 * [n][dim].
 * ------------------------------------------------------------------------ */
static int orc_collide_hit(const float *c, const float *r, int64_t dim, int64_t i, int64_t j)
{
    float s = 0.0f;
    for (int64_t k = 0; k < dim; ++k) {
        float dk = c[i * dim + k] - c[j * dim + k];
        float sq = dk * dk;
        s = k == 0 ? sq : s + sq;
    }
    float rr = r[i] + r[j];
    float rr2 = rr * rr;
    return s <= rr2;
}

/* hits[i - r0] = number of j < i colliding with sphere i, for r0 <= i < r1. */
void orc_collide_rows(const float *c, const float *r, int64_t dim, int64_t r0, int64_t r1, int64_t *hits)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = r0; i < r1; ++i) {
        int64_t h = 0;
        for (int64_t j = 0; j < i; ++j)
            h += orc_collide_hit(c, r, dim, i, j);
        hits[i - r0] = h;
    }
}

/* The colliding pairs of rows r0 <= i < r1 in increasing (i, j): row i writes
 * its pairs from position off[i - r0] (the exclusive prefix sum of the row
 * counts above). */
void orc_collide_pairs(const float *c, const float *r, int64_t dim, int64_t r0, int64_t r1, const int64_t *off,
                       uint32_t *pi, uint32_t *pj)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = r0; i < r1; ++i) {
        int64_t q = off[i - r0];
        for (int64_t j = 0; j < i; ++j)
            if (orc_collide_hit(c, r, dim, i, j)) {
                pi[q] = (uint32_t)i;
                pj[q] = (uint32_t)j;
                ++q;
            }
    }
}

/* For each listed sphere idx[t]: the number of other spheres it collides
 * with (both j < i and j > i), for sampled checks of per-sphere counts. */
void orc_collide_count_of(const float *c, const float *r, int64_t n, int64_t dim, const int64_t *idx, int64_t k,
                          int64_t *out)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < k; ++t) {
        int64_t i = idx[t], h = 0;
        for (int64_t j = 0; j < n; ++j)
            if (j != i)
                h += j < i ? orc_collide_hit(c, r, dim, i, j) : orc_collide_hit(c, r, dim, j, i);
        out[t] = h;
    }
}
