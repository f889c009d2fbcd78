/*
 * sph_oracle.c -- plain, slow CPU reference ("oracle") for the SPH hot path of
 * "The Shamrock code: I - Smoothed Particle Hydrodynamics on GPUs" (arXiv 2503.09713).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is used by the test-suite, by the smoke check and by the
 * CPU-baseline leg of the benchmark; the product library never calls, links or loads it.  It shares
 * no code, header, table or helper with the CUDA library.
 *
 * Conventions
 *   - FP64 everywhere; compiled with -ffp-contract=off so that no multiply-add is fused.
 *   - Every function names the passage of the paper it follows.  Where the paper is silent or
 *     garbled the reading taken is stated in the comment.
 *   - Functions that compute a quantity with a plain definition (Morton code, sort, radix tree,
 *     bounding boxes, neighbour set, root of the density equation) compute that definition
 *     directly.  Iterations (the smoothing-length update of App. F) follow the paper's steps.
 *   - OpenMP only parallelises independent per-particle loops; every reduction is a min or max,
 *     so results do not depend on the thread count.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* ====================================================================================== */
/* Morton codes: App. B, Sect. "Morton codes" (remap to [0,1)^3, (2^beta)^3 integer grid,   */
/* interleave X0 Y0 Z0 X1 Y1 Z1 ..., X most significant).                                   */
/* ====================================================================================== */

/* Integer grid coordinate of one axis: X = floor(((x - lo)/(hi - lo)) * 2^bits), clamped to
 * [0, 2^bits - 1] (the remap excludes 1, so a point on the upper face joins the last cell). */
uint64_t orc_quantise(double x, double lo, double hi, int bits)
{
    double s = (x - lo) / (hi - lo);
    double g = s * (double)(1ULL << bits); /* power-of-two scale: exact */
    double top = (double)((1ULL << bits) - 1ULL);
    if (!(g >= 0.0)) g = 0.0;
    if (g > top) g = top;
    return (uint64_t)floor(g);
}

/* Interleave three bits-wide integers bit by bit, most significant first: X0 Y0 Z0 X1 ... */
uint64_t orc_interleave(uint64_t X, uint64_t Y, uint64_t Z, int bits)
{
    uint64_t m = 0;
    for (int i = 0; i < bits; i++) {
        int b = bits - 1 - i;
        m = (m << 3) | (((X >> b) & 1ULL) << 2) | (((Y >> b) & 1ULL) << 1) | ((Z >> b) & 1ULL);
    }
    return m;
}

/* Inverse of orc_interleave (used only by the round-trip pin). */
void orc_deinterleave(uint64_t m, int bits, uint64_t *X, uint64_t *Y, uint64_t *Z)
{
    uint64_t x = 0, y = 0, z = 0;
    for (int i = 0; i < bits; i++) {
        int sh = 3 * (bits - 1 - i);
        x = (x << 1) | ((m >> (sh + 2)) & 1ULL);
        y = (y << 1) | ((m >> (sh + 1)) & 1ULL);
        z = (z << 1) | ((m >> sh) & 1ULL);
    }
    *X = x; *Y = y; *Z = z;
}

void orc_morton(int64_t n, const double *x, const double *y, const double *z,
                const double *lo, const double *hi, int bits, uint64_t *out)
{
    for (int64_t i = 0; i < n; i++)
        out[i] = orc_interleave(orc_quantise(x[i], lo[0], hi[0], bits),
                                orc_quantise(y[i], lo[1], hi[1], bits),
                                orc_quantise(z[i], lo[2], hi[2], bits), bits);
}

/* Length of the longest common prefix of two nbits-long codes, Eq. delta_ab: clz(a xor b),
 * counted within the nbits-wide representation. */
int orc_delta(uint64_t a, uint64_t b, int nbits)
{
    uint64_t v = a ^ b;
    if (v == 0) return nbits;
    int lz = 0;
    for (int k = 63; k >= 0; k--) {
        if ((v >> k) & 1ULL) break;
        lz++;
    }
    return lz - (64 - nbits);
}

/* ====================================================================================== */
/* Sort by key (App. C, "Sort by Key"): (code, original index) pairs ordered by code; equal   */
/* codes keep their original order, so the permutation is unique.                           */
/* ====================================================================================== */
typedef struct { uint64_t key; uint32_t idx; } orc_kv;

static int orc_kv_cmp(const void *pa, const void *pb)
{
    const orc_kv *a = (const orc_kv *)pa, *b = (const orc_kv *)pb;
    if (a->key < b->key) return -1;
    if (a->key > b->key) return 1;
    return (a->idx < b->idx) ? -1 : (a->idx > b->idx);
}

void orc_sort_by_key(int64_t n, const uint64_t *keys, uint64_t *sorted, uint32_t *perm)
{
    orc_kv *t = (orc_kv *)malloc((size_t)(n > 0 ? n : 1) * sizeof(orc_kv));
    for (int64_t i = 0; i < n; i++) { t[i].key = keys[i]; t[i].idx = (uint32_t)i; }
    qsort(t, (size_t)n, sizeof(orc_kv), orc_kv_cmp);
    for (int64_t i = 0; i < n; i++) { sorted[i] = t[i].key; perm[i] = t[i].idx; }
    free(t);
}

/* ====================================================================================== */
/* Keep mask and reduction (App. C, "Reduction").  Written from the criterion the appendix    */
/* states in words, not from its listing: duplicates are masked first (only the first of a    */
/* run of equal codes stays); then each reduction pass looks at the binary radix tree of the   */
/* codes kept so far and, for every internal node whose two children are both leaves, drops    */
/* the second (right) one of the two, so that pair of leaves becomes a single leaf.  The tree  */
/* is this file's own top-down construction (orc_radix_tree), a pass reads the tree of the     */
/* previous pass's result only (the paper's in-place parallel update is a race; reading: one   */
/* pass after the other), and the first code is never dropped (it is always a left child).    */
/* ====================================================================================== */
void orc_radix_tree(int64_t L, const uint64_t *mu_leaf, int nbits, int32_t *lchild, int32_t *rchild,
                    uint8_t *lflag, uint8_t *rflag, int32_t *endrange);

void orc_keep_mask(int64_t n, const uint64_t *mu, int nbits, int n_red, uint8_t *xi)
{
    if (n <= 0) return;
    for (int64_t i = 0; i < n; i++) xi[i] = (i == 0) ? 1 : (mu[i] != mu[i - 1]);
    int64_t *kept = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    uint64_t *codes = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    int32_t *lc = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *rc = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *er = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    uint8_t *lf = (uint8_t *)malloc((size_t)n);
    uint8_t *rf = (uint8_t *)malloc((size_t)n);
    for (int pass = 0; pass < n_red; pass++) {
        int64_t L = 0;
        for (int64_t i = 0; i < n; i++)
            if (xi[i]) { kept[L] = i; codes[L] = mu[i]; L++; }
        if (L < 2) break;
        orc_radix_tree(L, codes, nbits, lc, rc, lf, rf, er);
        for (int64_t c = 0; c < L - 1; c++)
            if (lf[c] && rf[c]) xi[kept[rc[c]]] = 0;   /* the second leaf of a leaf-leaf pair */
    }
    free(kept); free(codes); free(lc); free(rc); free(er); free(lf); free(rf);
}

/* Stream compaction (App. C, "Reduction"; Fig. mortonlistbuild): id[j] = index of the j-th kept
 * code, id[L] = n; mu_leaf[j] = mu[id[j]].  Returns L. */
int64_t orc_compact(int64_t n, const uint64_t *mu, const uint8_t *xi, int64_t *id, uint64_t *mu_leaf)
{
    int64_t L = 0;
    for (int64_t i = 0; i < n; i++)
        if (xi[i]) { id[L] = i; mu_leaf[L] = mu[i]; L++; }
    id[L] = n;
    return L;
}

/* ====================================================================================== */
/* Binary radix tree (App. B, "Binary radix tree" and "Karras algorithm", Table            */
/* arrays_fig_karras).  Built here by its definition, top-down: the node over leaves          */
/* [first,last] splits after the last leaf that shares with leaf `first` a prefix longer than */
/* delta(first,last).  The left child covers [first,g], the right child [g+1,last]; a child   */
/* over one leaf is that leaf (flag 1), otherwise it is the internal node whose index is the  */
/* end of its range next to the split (g for the left child, g+1 for the right child); the    */
/* root is internal node 0.  endrange holds the other end of each internal node's range.     */
/* ====================================================================================== */
static void orc_split(const uint64_t *mu, int nbits, int64_t node, int64_t first, int64_t last,
                      int32_t *lchild, int32_t *rchild, uint8_t *lflag, uint8_t *rflag, int32_t *endrange)
{
    int d = orc_delta(mu[first], mu[last], nbits);
    int64_t g = first;
    for (int64_t k = first + 1; k < last; k++)
        if (orc_delta(mu[first], mu[k], nbits) > d) g = k;
    endrange[node] = (int32_t)((node == first) ? last : first);
    lchild[node] = (int32_t)g;
    lflag[node] = (g == first);
    rchild[node] = (int32_t)(g + 1);
    rflag[node] = (g + 1 == last);
    if (g != first) orc_split(mu, nbits, g, first, g, lchild, rchild, lflag, rflag, endrange);
    if (g + 1 != last) orc_split(mu, nbits, g + 1, g + 1, last, lchild, rchild, lflag, rflag, endrange);
}

/* mu_leaf: L sorted distinct codes.  Fills L-1 internal nodes. */
void orc_radix_tree(int64_t L, const uint64_t *mu_leaf, int nbits, int32_t *lchild, int32_t *rchild,
                    uint8_t *lflag, uint8_t *rflag, int32_t *endrange)
{
    if (L < 2) return;
    orc_split(mu_leaf, nbits, 0, 0, L - 1, lchild, rchild, lflag, rflag, endrange);
}

/* Tight bounding box and largest smoothing length of every tree cell (App. C, "Compute tree cell
 * sizes"; the h_max per cell is l_AABB,b of App. D).  Nodes 0..L-2 are internal, node L-1+j is
 * leaf j.  A cell's particles are the sorted positions id[first] .. id[last+1]-1 of its leaf range.
 * Positions/h are given in sorted order. */
void orc_cell_boxes(int64_t L, const int64_t *id, const int32_t *endrange,
                    const double *x, const double *y, const double *z, const double *h,
                    double *bmin /*3*(2L-1)*/, double *bmax, double *hmax /*2L-1*/)
{
    int64_t nodes = 2 * L - 1;
    for (int64_t c = 0; c < nodes; c++) {
        int64_t first, last;
        if (c < L - 1) {
            int64_t e = endrange[c];
            first = c < e ? c : e;
            last = c < e ? e : c;
        } else {
            first = last = c - (L - 1);
        }
        double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
        double hm = 0.0;
        for (int64_t p = id[first]; p < id[last + 1]; p++) {
            double r[3] = {x[p], y[p], z[p]};
            for (int k = 0; k < 3; k++) {
                if (r[k] < mn[k]) mn[k] = r[k];
                if (r[k] > mx[k]) mx[k] = r[k];
            }
            if (h[p] > hm) hm = h[p];
        }
        for (int k = 0; k < 3; k++) { bmin[3 * c + k] = mn[k]; bmax[3 * c + k] = mx[k]; }
        hmax[c] = hm;
    }
}

/* ====================================================================================== */
/* M4 cubic spline (Sect. 2.1: B-spline M4, 3-D normalisation).  Reading: Schoenberg M4 as in  */
/* Monaghan & Lattanzio 1985, f(q) = 1 - 3/2 q^2 + 3/4 q^3 (q<1), (2-q)^3/4 (1<=q<2), 0 after,   */
/* C_norm = 1/pi, R_kern = 2.  W = C_norm f(q)/h^3 (Eq. rhosphsum), q = r/h.                   */
/* ====================================================================================== */
double orc_m4_f(double q)
{
    if (q < 1.0) return 1.0 - 1.5 * q * q + 0.75 * q * q * q;
    if (q < 2.0) { double t = 2.0 - q; return 0.25 * t * t * t; }
    return 0.0;
}

double orc_m4_df(double q) /* df/dq */
{
    if (q < 1.0) return -3.0 * q + 2.25 * q * q;
    if (q < 2.0) { double t = 2.0 - q; return -0.75 * t * t; }
    return 0.0;
}

/* ====================================================================================== */
/* The other kernels of Sect. 2.1 ("B-splines like M4, M5, M6, or Wendland functions like C2, */
/* C4, C6"), each as its textbook piecewise definition on q = r/h with its support R_kern and  */
/* its 3-D normalisation C_norm (4 pi C_norm int_0^R f q^2 dq = 1):                            */
/*   M5 (R 5/2, C 1/(20 pi)):  (5/2-q)^4 - 5 (3/2-q)^4 + 10 (1/2-q)^4 on [0,1/2), dropping the  */
/*      last and then the middle term on [1/2,3/2) and [3/2,5/2)                               */
/*   M6 (R 3, C 1/(120 pi)):  (3-q)^5 - 6 (2-q)^5 + 15 (1-q)^5 on [0,1), likewise              */
/*   Wendland (R 2):  C2 = (1-q/2)^4 (1+2q), C 21/(16 pi);  C4 = (1-q/2)^6 (1+3q+35/12 q^2),    */
/*      C 495/(256 pi);  C6 = (1-q/2)^8 (1+4q+25/4 q^2+4q^3), C 1365/(512 pi)                   */
/* The kernel in use is a module setting (orc_set_kernel; 0 = M4, 1 = M5, 2 = M6, 3 = C2,       */
/* 4 = C4, 5 = C6), read by every function below.                                              */
/* ====================================================================================== */
static int orc_kind = 0;

void orc_set_kernel(int kind) { orc_kind = kind; }

double orc_kernel_R(int kind)
{
    if (kind == 1) return 2.5;
    if (kind == 2) return 3.0;
    return 2.0;
}

double orc_kernel_C(int kind)
{
    switch (kind) {
    case 1: return 1.0 / (20.0 * ORC_PI);
    case 2: return 1.0 / (120.0 * ORC_PI);
    case 3: return 21.0 / (16.0 * ORC_PI);
    case 4: return 495.0 / (256.0 * ORC_PI);
    case 5: return 1365.0 / (512.0 * ORC_PI);
    default: return 1.0 / ORC_PI;
    }
}

static double p4(double v) { return v * v * v * v; }
static double p5(double v) { return v * v * v * v * v; }

double orc_kernel_f(int kind, double q)
{
    double w = 1.0 - 0.5 * q;
    switch (kind) {
    case 1:
        if (q < 0.5) return p4(2.5 - q) - 5.0 * p4(1.5 - q) + 10.0 * p4(0.5 - q);
        if (q < 1.5) return p4(2.5 - q) - 5.0 * p4(1.5 - q);
        if (q < 2.5) return p4(2.5 - q);
        return 0.0;
    case 2:
        if (q < 1.0) return p5(3.0 - q) - 6.0 * p5(2.0 - q) + 15.0 * p5(1.0 - q);
        if (q < 2.0) return p5(3.0 - q) - 6.0 * p5(2.0 - q);
        if (q < 3.0) return p5(3.0 - q);
        return 0.0;
    case 3:
        if (q < 2.0) return pow(w, 4.0) * (1.0 + 2.0 * q);
        return 0.0;
    case 4:
        if (q < 2.0) return pow(w, 6.0) * (1.0 + 3.0 * q + 35.0 / 12.0 * q * q);
        return 0.0;
    case 5:
        if (q < 2.0) return pow(w, 8.0) * (1.0 + 4.0 * q + 25.0 / 4.0 * q * q + 4.0 * q * q * q);
        return 0.0;
    default:
        return orc_m4_f(q);
    }
}

/* df/dq, differentiated term by term (chain and product rules as written, not simplified). */
double orc_kernel_df(int kind, double q)
{
    double w = 1.0 - 0.5 * q;
    switch (kind) {
    case 1: {
        double d = 0.0;
        if (q < 2.5) d += -4.0 * pow(2.5 - q, 3.0);
        if (q < 1.5) d += 20.0 * pow(1.5 - q, 3.0);
        if (q < 0.5) d += -40.0 * pow(0.5 - q, 3.0);
        return d;
    }
    case 2: {
        double d = 0.0;
        if (q < 3.0) d += -5.0 * p4(3.0 - q);
        if (q < 2.0) d += 30.0 * p4(2.0 - q);
        if (q < 1.0) d += -75.0 * p4(1.0 - q);
        return d;
    }
    case 3:
        if (q < 2.0) return 4.0 * pow(w, 3.0) * (-0.5) * (1.0 + 2.0 * q) + pow(w, 4.0) * 2.0;
        return 0.0;
    case 4:
        if (q < 2.0)
            return 6.0 * pow(w, 5.0) * (-0.5) * (1.0 + 3.0 * q + 35.0 / 12.0 * q * q) +
                   pow(w, 6.0) * (3.0 + 35.0 / 6.0 * q);
        return 0.0;
    case 5:
        if (q < 2.0)
            return 8.0 * pow(w, 7.0) * (-0.5) * (1.0 + 4.0 * q + 25.0 / 4.0 * q * q + 4.0 * q * q * q) +
                   pow(w, 8.0) * (4.0 + 25.0 / 2.0 * q + 12.0 * q * q);
        return 0.0;
    default:
        return orc_m4_df(q);
    }
}

double orc_W(double r, double h) { return orc_kernel_C(orc_kind) * orc_kernel_f(orc_kind, r / h) / (h * h * h); }

/* dW/dh at fixed r. */
double orc_dWdh(double r, double h)
{
    double q = r / h;
    return -orc_kernel_C(orc_kind) * (3.0 * orc_kernel_f(orc_kind, q) + q * orc_kernel_df(orc_kind, q)) /
           (h * h * h * h);
}

/* F_ab(h) = rhat . grad_a W_ab(h) = dW/dr (Sect. 2.1 definition of F_ab). */
double orc_F(double r, double h) { return orc_kernel_C(orc_kind) * orc_kernel_df(orc_kind, r / h) / (h * h * h * h); }

/* ====================================================================================== */
/* Neighbour sets (App. D criteria, App. C neighbour caches).                                */
/* A pair (a,b), b != a, belongs to the set at radius scale s when                           */
/*     r_ab^2 < (s * max(hc_a, hc_b))^2                                                       */
/* with r_ab^2 = (dx*dx + dy*dy) + dz*dz evaluated in that order, dx = x_b - x_a reduced to the */
/* nearest periodic image (dx > L/2: dx -= L; dx < -L/2: dx += L).  s = R_kern * chi for the  */
/* cache (App. F tolerance chi), s = R_kern for the force support (object-object criterion).  */
/* ====================================================================================== */
typedef struct {
    int64_t n;
    int64_t *off; /* n+1 */
    int32_t *ids; /* off[n] entries, each list ascending in b */
} orc_nlist;

static double orc_image(double d, double L, int periodic)
{
    if (periodic) {
        if (d > 0.5 * L) d -= L;
        else if (d < -0.5 * L) d += L;
    }
    return d;
}

static int orc_pair_in(const double *x, const double *y, const double *z, const double *hc,
                       int64_t a, int64_t b, double s, const double *boxL, int periodic)
{
    double dx = orc_image(x[b] - x[a], boxL[0], periodic);
    double dy = orc_image(y[b] - y[a], boxL[1], periodic);
    double dz = orc_image(z[b] - z[a], boxL[2], periodic);
    double r2 = (dx * dx + dy * dy) + dz * dz;
    double hm = hc[a] > hc[b] ? hc[a] : hc[b];
    double rad = s * hm;
    return r2 < rad * rad;
}

/* Direct O(N^2) evaluation of the definition. */
static void orc_nlist_brute(int64_t n, const double *x, const double *y, const double *z, const double *hc,
                            double s, const double *boxL, int periodic, orc_nlist *nl)
{
    nl->n = n;
    nl->off = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    int64_t *cnt = (int64_t *)calloc((size_t)(n + 1), sizeof(int64_t));
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t a = 0; a < n; a++) {
        int64_t c = 0;
        for (int64_t b = 0; b < n; b++)
            if (b != a && orc_pair_in(x, y, z, hc, a, b, s, boxL, periodic)) c++;
        cnt[a] = c;
    }
    nl->off[0] = 0;
    for (int64_t a = 0; a < n; a++) nl->off[a + 1] = nl->off[a] + cnt[a];
    nl->ids = (int32_t *)malloc((size_t)(nl->off[n] > 0 ? nl->off[n] : 1) * sizeof(int32_t));
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t a = 0; a < n; a++) {
        int64_t o = nl->off[a];
        for (int64_t b = 0; b < n; b++)
            if (b != a && orc_pair_in(x, y, z, hc, a, b, s, boxL, periodic)) nl->ids[o++] = (int32_t)b;
    }
    free(cnt);
}

/* Same set through a uniform grid of cells no smaller than the largest radius: only particles in
 * the 27 surrounding cells can satisfy the predicate, which is then evaluated exactly as above and
 * the survivors listed in ascending index order.  Used for sizes beyond brute force; tests check it
 * against orc_nlist_brute. */
static int orc_cmp_i32(const void *a, const void *b)
{
    int32_t u = *(const int32_t *)a, v = *(const int32_t *)b;
    return (u > v) - (u < v);
}

static void orc_nlist_grid(int64_t n, const double *x, const double *y, const double *z, const double *hc,
                           double s, const double *lo, const double *boxL, int periodic, orc_nlist *nl)
{
    double hmax = 0.0;
    for (int64_t i = 0; i < n; i++) if (hc[i] > hmax) hmax = hc[i];
    double rmax = s * hmax;
    int64_t nc[3];
    for (int k = 0; k < 3; k++) {
        double c = floor(boxL[k] / rmax);
        if (c > 256) c = 256;
        nc[k] = (int64_t)c;
    }
    if (nc[0] < 3 || nc[1] < 3 || nc[2] < 3 || n < 2048) {
        orc_nlist_brute(n, x, y, z, hc, s, boxL, periodic, nl);
        return;
    }
    int64_t ncell = nc[0] * nc[1] * nc[2];
    int64_t *cell = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *head = (int64_t *)calloc((size_t)(ncell + 1), sizeof(int64_t));
    int64_t *order = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    const double *pos[3] = {x, y, z};
    for (int64_t i = 0; i < n; i++) {
        int64_t ci[3];
        for (int k = 0; k < 3; k++) {
            int64_t c = (int64_t)floor((pos[k][i] - lo[k]) / boxL[k] * (double)nc[k]);
            if (c < 0) c = 0;
            if (c >= nc[k]) c = nc[k] - 1;
            ci[k] = c;
        }
        cell[i] = (ci[0] * nc[1] + ci[1]) * nc[2] + ci[2];
        head[cell[i] + 1]++;
    }
    for (int64_t c = 0; c < ncell; c++) head[c + 1] += head[c];
    int64_t *fill = (int64_t *)malloc((size_t)ncell * sizeof(int64_t));
    memcpy(fill, head, (size_t)ncell * sizeof(int64_t));
    for (int64_t i = 0; i < n; i++) order[fill[cell[i]]++] = i;
    free(fill);

    nl->n = n;
    nl->off = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    int64_t *cnt = (int64_t *)calloc((size_t)(n + 1), sizeof(int64_t));
    for (int pass = 0; pass < 2; pass++) {
        if (pass == 1) {
            nl->off[0] = 0;
            for (int64_t a = 0; a < n; a++) nl->off[a + 1] = nl->off[a] + cnt[a];
            nl->ids = (int32_t *)malloc((size_t)(nl->off[n] > 0 ? nl->off[n] : 1) * sizeof(int32_t));
        }
#pragma omp parallel for schedule(dynamic, 256)
        for (int64_t a = 0; a < n; a++) {
            int64_t c = cell[a];
            int64_t cz = c % nc[2], cy = (c / nc[2]) % nc[1], cx = c / (nc[1] * nc[2]);
            int64_t o = (pass == 1) ? nl->off[a] : 0;
            int64_t k = 0;
            for (int ox = -1; ox <= 1; ox++)
                for (int oy = -1; oy <= 1; oy++)
                    for (int oz = -1; oz <= 1; oz++) {
                        int64_t qx = cx + ox, qy = cy + oy, qz = cz + oz;
                        if (periodic) {
                            qx = (qx + nc[0]) % nc[0]; qy = (qy + nc[1]) % nc[1]; qz = (qz + nc[2]) % nc[2];
                        } else if (qx < 0 || qy < 0 || qz < 0 || qx >= nc[0] || qy >= nc[1] || qz >= nc[2]) {
                            continue;
                        }
                        int64_t q = (qx * nc[1] + qy) * nc[2] + qz;
                        for (int64_t t = head[q]; t < head[q + 1]; t++) {
                            int64_t b = order[t];
                            if (b != a && orc_pair_in(x, y, z, hc, a, b, s, boxL, periodic)) {
                                if (pass == 1) nl->ids[o + k] = (int32_t)b;
                                k++;
                            }
                        }
                    }
            if (pass == 0) cnt[a] = k;
            else qsort(nl->ids + o, (size_t)k, sizeof(int32_t), orc_cmp_i32);
        }
    }
    free(cnt); free(cell); free(head); free(order);
}

static void orc_nlist_free(orc_nlist *nl)
{
    free(nl->off); free(nl->ids);
    nl->off = NULL; nl->ids = NULL;
}

/* Exported neighbour-set builder.  method 0 = brute force, 1 = grid.  Returns the pair count and,
 * when off/ids are non-NULL, copies the lists out (ids must hold the returned count). */
static orc_nlist orc_last_list = {0, NULL, NULL};

int64_t orc_neighbours(int64_t n, const double *x, const double *y, const double *z, const double *hc,
                       double s, const double *lo, const double *hi, int periodic, int method)
{
    double boxL[3] = {hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]};
    orc_nlist_free(&orc_last_list);
    if (method == 0) orc_nlist_brute(n, x, y, z, hc, s, boxL, periodic, &orc_last_list);
    else orc_nlist_grid(n, x, y, z, hc, s, lo, boxL, periodic, &orc_last_list);
    return orc_last_list.off[n];
}

void orc_neighbours_copy(int64_t *off, int32_t *ids)
{
    int64_t n = orc_last_list.n;
    memcpy(off, orc_last_list.off, (size_t)(n + 1) * sizeof(int64_t));
    memcpy(ids, orc_last_list.ids, (size_t)orc_last_list.off[n] * sizeof(int32_t));
}

/* ====================================================================================== */
/* Parameters of the hydrodynamics (Sect. 2.1, App. F, App. G).                              */
/* ====================================================================================== */
typedef struct {
    double hfact;     /* rho(h) = m (hfact/h)^3, Eq. rhoh */
    double gamma;     /* adiabatic index: P = (gamma-1) rho u */
    double alpha_av;  /* alpha^AV in v_sig */
    double beta_av;   /* beta in v_sig */
    double alpha_u;   /* beta_u of Lambda_cond (0 switches conductivity off) */
    double c_cour, c_force; /* CFL safety factors, App. G */
    double h_tol;     /* epsilon_c of App. F */
    double h_clamp;   /* lambda of App. F */
    double cache_tol; /* chi of App. F */
    double lo[3], hi[3];
    int periodic;
    int h_max_iter;
    /* shock switch, CFL multiplier and corrector re-runs (App. G "CFL multiplier", "Shock
     * detection"); av_switch = 0 and eps_v = 0 give the fixed-alpha step above */
    int av_switch;       /* 1: alpha_a evolves (Eq. evolalphaanalytic), alpha_av is alpha_max */
    int max_corr;        /* most corrector passes per step */
    double alpha_min;    /* floor of alpha_loc */
    double sigma_decay;  /* tau_a = h_a / (sigma_decay c_s,a) */
    double eps_v;        /* epsilon_v of Eq. cvleapfrog; 0: no re-run */
    double lambda_stiff; /* lambda_stiff of the CFL multiplier recovery */
} orc_params;

static double orc_dist(const double *x, const double *y, const double *z, int64_t a, int64_t b,
                       const double *boxL, int periodic, double *d /*3, r_a - r_b*/)
{
    d[0] = orc_image(x[a] - x[b], boxL[0], periodic);
    d[1] = orc_image(y[a] - y[b], boxL[1], periodic);
    d[2] = orc_image(z[a] - z[b], boxL[2], periodic);
    return sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]);
}

/* SPH density sum and its h-derivative for particle a at trial h (Eq. SPHmass / rhosphsum), the
 * sum running over the cached candidates and a itself (r = 0). */
static void orc_rho_sums(int64_t a, double h, double mass, const orc_nlist *nl,
                         const double *x, const double *y, const double *z, const double *boxL, int periodic,
                         double *rho_sum, double *drho_dh)
{
    double s0 = mass * orc_W(0.0, h), s1 = mass * orc_dWdh(0.0, h);
    for (int64_t k = nl->off[a]; k < nl->off[a + 1]; k++) {
        int64_t b = nl->ids[k];
        double d[3];
        double r = orc_dist(x, y, z, a, b, boxL, periodic, d);
        if (r < orc_kernel_R(orc_kind) * h) {
            s0 += mass * orc_W(r, h);
            s1 += mass * orc_dWdh(r, h);
        }
    }
    *rho_sum = s0;
    *drho_dh = s1;
}

/* ---------------------------------------------------------------------------------------- */
/* Root of the density equation, by its definition (App. F, Eq. rhoh with Eq. SPHmass):       */
/* h_a solves  sum_b m W(r_ab, h_a) = m (hfact/h_a)^3.  h^3 * sum_b W is non-decreasing in h   */
/* (f is non-increasing in q), so the root is unique and bisection on                          */
/*      phi(h) = sum_b f(r_ab/h)/pi - hfact^3                                                 */
/* brackets it.  Candidates: every b within R_kern * h_hi (brute force or grid).              */
/* ---------------------------------------------------------------------------------------- */
static double orc_phi(int64_t a, double h, const orc_nlist *nl, const double *x, const double *y,
                      const double *z, const double *boxL, int periodic, double hfact)
{
    double C = orc_kernel_C(orc_kind);
    double s = C * orc_kernel_f(orc_kind, 0.0);
    for (int64_t k = nl->off[a]; k < nl->off[a + 1]; k++) {
        double d[3];
        double r = orc_dist(x, y, z, a, nl->ids[k], boxL, periodic, d);
        s += C * orc_kernel_f(orc_kind, r / h);
    }
    return s - hfact * hfact * hfact;
}

/* h_hi: an upper bracket for every particle (phi(h_hi) > 0 is checked; returns the number of
 * particles whose bracket failed, which are left at NaN). */
int64_t orc_density_root(int64_t n, const double *x, const double *y, const double *z,
                         double hfact, double h_hi, const double *lo, const double *hi, int periodic,
                         int method, double *h_out)
{
    double boxL[3] = {hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]};
    double *hc = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    for (int64_t i = 0; i < n; i++) hc[i] = h_hi;
    orc_nlist nl;
    double R = orc_kernel_R(orc_kind);
    if (method == 0) orc_nlist_brute(n, x, y, z, hc, R, boxL, periodic, &nl);
    else orc_nlist_grid(n, x, y, z, hc, R, lo, boxL, periodic, &nl);
    int64_t bad = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : bad)
    for (int64_t a = 0; a < n; a++) {
        double hl = 0.0, hh = h_hi;
        if (!(orc_phi(a, hh, &nl, x, y, z, boxL, periodic, hfact) > 0.0)) { h_out[a] = NAN; bad++; continue; }
        /* lower bracket: h below half the nearest distance sees only the self term, phi < 0 */
        for (int it = 0; it < 200; it++) {
            double hm = 0.5 * (hl + hh);
            if (hm <= hl || hm >= hh) break;
            if (hl > 0.0 && (hh - hl) <= 1e-16 * hh) break;
            if (orc_phi(a, hm, &nl, x, y, z, boxL, periodic, hfact) > 0.0) hh = hm;
            else hl = hm;
        }
        h_out[a] = 0.5 * (hl + hh);
    }
    orc_nlist_free(&nl);
    free(hc);
    return bad;
}

/* ---------------------------------------------------------------------------------------- */
/* Smoothing-length update, Alg. "Smoothing length update" (App. F), in the paper's order:     */
/*   outer loop: build the candidate lists at R_kern * chi * max(h_a^n, h_b^n) (the ghost /     */
/*     cache tolerance), inner Newton-Raphson loop on delta rho = rho_a - rho(h_a):            */
/*       d(delta rho) = sum_b m dW/dh + 3 rho(h_a)/h_a          (reading: the analytic         */
/*                                                               derivative, rho(h) of Eq. rhoh) */
/*       h <- h - delta rho / d(delta rho), clamped to [h/lambda, h*lambda]                     */
/*       eps_a = |h_new - h| / h_a^n; h_new > chi h_a^n -> h_new = chi h_a^n, eps_a = -1           */
/*   until max eps <= eps_c; restart the outer loop while some eps = -1, with h^n := current h  */
/*   (reading of "restart with the updated smoothing length").                                  */
/* Epilogue: rho_a = rho(h_a) (Eq. rhoh), Omega_a = 1 - (dh/drho) sum_b m dW/dh with             */
/* dh/drho = -h/(3 rho) (Eq. sphomega), evaluated at the final h.                                */
/* Returns total inner iterations (>= 0) or -1 when h_max_iter was exceeded.  outer_out: the    */
/* number of outer passes.                                                                      */
/* ---------------------------------------------------------------------------------------- */
int orc_density_algF(int64_t n, double mass, const orc_params *p, const double *x, const double *y,
                     const double *z, double *h, double *rho, double *omega, int method, int *outer_out)
{
    double boxL[3] = {p->hi[0] - p->lo[0], p->hi[1] - p->lo[1], p->hi[2] - p->lo[2]};
    double *hn = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    double *eps = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    double *hnew = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    int total = 0, outer = 0, failed = 0;
    for (int64_t a = 0; a < n; a++) eps[a] = -1.0;
    double mineps = -1.0;
    while (mineps == -1.0 && n > 0) {
        outer++;
        for (int64_t a = 0; a < n; a++) hn[a] = h[a];
        orc_nlist nl;
        double s = orc_kernel_R(orc_kind) * p->cache_tol;
        if (method == 0) orc_nlist_brute(n, x, y, z, hn, s, boxL, p->periodic, &nl);
        else orc_nlist_grid(n, x, y, z, hn, s, p->lo, boxL, p->periodic, &nl);
        double maxeps = INFINITY;
        while (maxeps > p->h_tol) {
            if (total >= p->h_max_iter) { failed = 1; break; }
            total++;
#pragma omp parallel for schedule(dynamic, 64)
            for (int64_t a = 0; a < n; a++) {
                double ha = h[a];
                double rs, ds;
                orc_rho_sums(a, ha, mass, &nl, x, y, z, boxL, p->periodic, &rs, &ds);
                double rho_h = mass * pow(p->hfact / ha, 3.0);
                double drho = rs - rho_h;
                double ddrho = ds + 3.0 * rho_h / ha;
                double hnw = ha - drho / ddrho;
                if (hnw > ha * p->h_clamp) hnw = ha * p->h_clamp;
                else if (hnw < ha / p->h_clamp) hnw = ha / p->h_clamp;
                double e = fabs(hnw - ha) / hn[a];
                if (hnw > hn[a] * p->cache_tol) { hnw = hn[a] * p->cache_tol; e = -1.0; }
                hnew[a] = hnw;
                eps[a] = e;
            }
            maxeps = -INFINITY;
            mineps = INFINITY;
            for (int64_t a = 0; a < n; a++) {
                h[a] = hnew[a];
                if (eps[a] > maxeps) maxeps = eps[a];
                if (eps[a] < mineps) mineps = eps[a];
            }
        }
        if (!failed) {
            mineps = INFINITY;
            for (int64_t a = 0; a < n; a++) if (eps[a] < mineps) mineps = eps[a];
        }
        if (failed) { orc_nlist_free(&nl); break; }
        if (mineps != -1.0) {
#pragma omp parallel for schedule(dynamic, 64)
            for (int64_t a = 0; a < n; a++) {
                double rs, ds;
                orc_rho_sums(a, h[a], mass, &nl, x, y, z, boxL, p->periodic, &rs, &ds);
                double rho_h = mass * pow(p->hfact / h[a], 3.0);
                rho[a] = rho_h;
                omega[a] = 1.0 + h[a] / (3.0 * rho_h) * ds;
            }
        }
        orc_nlist_free(&nl);
    }
    free(hn); free(eps); free(hnew);
    if (outer_out) *outer_out = outer;
    return failed ? -1 : total;
}

/* Density and Omega at given smoothing lengths (no iteration): rho_sum_a (Eq. SPHmass) and
 * Omega_a (Eq. sphomega with rho = rho(h_a)).  Used by pins on h-independent quantities. */
void orc_density_at(int64_t n, double mass, double hfact, const double *x, const double *y, const double *z,
                    const double *h, const double *lo, const double *hi, int periodic, int method,
                    double *rho_sum, double *omega)
{
    double boxL[3] = {hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]};
    orc_nlist nl;
    double R = orc_kernel_R(orc_kind);
    if (method == 0) orc_nlist_brute(n, x, y, z, h, R, boxL, periodic, &nl);
    else orc_nlist_grid(n, x, y, z, h, R, lo, boxL, periodic, &nl);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t a = 0; a < n; a++) {
        double rs, ds;
        orc_rho_sums(a, h[a], mass, &nl, x, y, z, boxL, periodic, &rs, &ds);
        double rho_h = mass * pow(hfact / h[a], 3.0);
        rho_sum[a] = rs;
        omega[a] = 1.0 + h[a] / (3.0 * rho_h) * ds;
    }
    orc_nlist_free(&nl);
}

/* ====================================================================================== */
/* Derivatives (Sect. 2.1, Eqs. sphvel, sphuint, q^a_ab, v_sig, Lambda_cond, F_ab).          */
/* Readings:                                                                                */
/*   - dv_a/dt carries a minus sign: a_a = -sum_b m [(P_a+q^a)/(rho_a^2 Omega_a) grad_a W(h_a) */
/*     + (P_b+q^b)/(rho_b^2 Omega_b) grad_a W(h_b)]; the printed form has none, which would make */
/*     pressure attractive and break energy conservation.                                     */
/*   - q^a_ab sits inside the sum of Eq. sphuint: du_a/dt = sum_b m (P_a+q^a_ab)/(rho_a^2      */
/*     Omega_a) v_ab . grad_a W_ab(h_a) + Lambda_cond.                                         */
/*   - grad_a W_ab(h) = rhat_ab F_ab(h), rhat_ab = (r_a - r_b)/|r_a - r_b|.                     */
/*   - pairs interact when r_ab < R_kern max(h_a, h_b) (object-object criterion, App. D).      */
/*   - v_sig^dt_a = max_b (alpha c_s,a + beta max(0, -v_ab . rhat_ab)), alpha c_s,a without     */
/*     neighbours (the paper does not define v_sig^dt).                                       */
/*   - rho_a = rho(h_a) (Eq. rhoh), P_a = (gamma-1) rho_a u_a, c_s,a = sqrt(gamma P_a/rho_a).   */
/* Inputs are per-particle h, Omega (rho follows from h); outputs ax,ay,az,du,vsig.           */
/* ====================================================================================== */
void orc_forces_alpha(int64_t n, double mass, const orc_params *p, const double *x, const double *y,
                      const double *z, const double *vx, const double *vy, const double *vz, const double *u,
                      const double *h, const double *omega, const double *alpha, int method,
                      double *ax, double *ay, double *az, double *du, double *vsig)
{
    double boxL[3] = {p->hi[0] - p->lo[0], p->hi[1] - p->lo[1], p->hi[2] - p->lo[2]};
    double *rho = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    double *P = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    double *cs = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    for (int64_t a = 0; a < n; a++) {
        rho[a] = mass * pow(p->hfact / h[a], 3.0);
        P[a] = (p->gamma - 1.0) * rho[a] * u[a];
        cs[a] = sqrt(p->gamma * P[a] / rho[a]);
    }
    orc_nlist nl;
    double R = orc_kernel_R(orc_kind);
    if (method == 0) orc_nlist_brute(n, x, y, z, h, R, boxL, p->periodic, &nl);
    else orc_nlist_grid(n, x, y, z, h, R, p->lo, boxL, p->periodic, &nl);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t a = 0; a < n; a++) {
        double acc[3] = {0.0, 0.0, 0.0}, dua = 0.0;
        double al_a = alpha ? alpha[a] : p->alpha_av;
        double vs = al_a * cs[a];
        for (int64_t k = nl.off[a]; k < nl.off[a + 1]; k++) {
            int64_t b = nl.ids[k];
            double d[3];
            double r = orc_dist(x, y, z, a, b, boxL, p->periodic, d);
            double rhat[3] = {d[0] / r, d[1] / r, d[2] / r};
            double vab[3] = {vx[a] - vx[b], vy[a] - vy[b], vz[a] - vz[b]};
            double vdotr = vab[0] * rhat[0] + vab[1] * rhat[1] + vab[2] * rhat[2];
            double Fa = orc_F(r, h[a]);
            double Fb = orc_F(r, h[b]);
            double qa = 0.0, qb = 0.0;
            double al_b = alpha ? alpha[b] : p->alpha_av;
            if (vdotr < 0.0) {
                double vsa = al_a * cs[a] + p->beta_av * fabs(vdotr);
                double vsb = al_b * cs[b] + p->beta_av * fabs(vdotr);
                qa = -0.5 * rho[a] * vsa * vdotr;
                qb = -0.5 * rho[b] * vsb * vdotr;
            }
            double Aa = (P[a] + qa) / (rho[a] * rho[a] * omega[a]);
            double Ab = (P[b] + qb) / (rho[b] * rho[b] * omega[b]);
            double sc = mass * (Aa * Fa + Ab * Fb);
            for (int c = 0; c < 3; c++) acc[c] -= sc * rhat[c];
            dua += mass * Aa * vdotr * Fa;
            if (p->alpha_u != 0.0) {
                double vsu = sqrt(fabs(P[a] - P[b]) / (0.5 * (rho[a] + rho[b])));
                dua += mass * p->alpha_u * vsu * (u[a] - u[b]) * 0.5 *
                       (Fa / (omega[a] * rho[a]) + Fb / (omega[b] * rho[b]));
            }
            double vsdt = al_a * cs[a] + p->beta_av * (vdotr < 0.0 ? -vdotr : 0.0);
            if (vsdt > vs) vs = vsdt;
        }
        ax[a] = acc[0]; ay[a] = acc[1]; az[a] = acc[2];
        du[a] = dua;
        vsig[a] = vs;
    }
    orc_nlist_free(&nl);
    free(rho); free(P); free(cs);
}

/* Fixed alpha = alpha_av for every particle. */
void orc_forces(int64_t n, double mass, const orc_params *p, const double *x, const double *y,
                const double *z, const double *vx, const double *vy, const double *vz, const double *u,
                const double *h, const double *omega, int method,
                double *ax, double *ay, double *az, double *du, double *vsig)
{
    orc_forces_alpha(n, mass, p, x, y, z, vx, vy, vz, u, h, omega, NULL, method, ax, ay, az, du, vsig);
}

/* ====================================================================================== */
/* Shock detection (App. G, Eq. evolalphaanalytic and its implicit step; the paper refers to     */
/* Phantom, Price et al. 2018, Sect. 2.2.9, for the switch).  Reading:                           */
/*   velocity and acceleration gradients by the SPH estimator at h_a,                              */
/*     (d_j v^i)_a = -1/(Omega_a rho_a) sum_b m (v_a^i - v_b^i) F_ab(h_a) rhat_ab^j,  likewise a;   */
/*   d(div v)/dt = div a - (d_i v^j)(d_j v^i);                                                    */
/*   xi_a = |div v|^2 / (|div v|^2 + |curl v|^2)   (0 when both vanish);                           */
/*   A_a = xi_a max(-d(div v)/dt, 0);  alpha_loc = max(alpha_min, min(10 h_a^2 A_a / c_s,a^2,       */
/*   alpha_max));  tau_a = h_a / (sigma_decay c_s,a);                                              */
/*   alpha^{n+1} = max((alpha^n + alpha_loc dt/tau)/(1 + dt/tau), alpha_loc)  (the paper's step).  */
/* Evaluated after the predictor and the h iteration, with v* and a^n (alpha_loc(v*, grad v*,      */
/* grad a^n)) and c_s from u*; alpha_max = alpha_av.                                                */
/* ====================================================================================== */
void orc_alpha_update(int64_t n, double mass, const orc_params *p, const double *x, const double *y,
                      const double *z, const double *vx, const double *vy, const double *vz, const double *ax,
                      const double *ay, const double *az, const double *u, const double *h,
                      const double *omega, double dt, int method, double *alpha)
{
    double boxL[3] = {p->hi[0] - p->lo[0], p->hi[1] - p->lo[1], p->hi[2] - p->lo[2]};
    orc_nlist nl;
    double R = orc_kernel_R(orc_kind);
    if (method == 0) orc_nlist_brute(n, x, y, z, h, R, boxL, p->periodic, &nl);
    else orc_nlist_grid(n, x, y, z, h, R, p->lo, boxL, p->periodic, &nl);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t a = 0; a < n; a++) {
        double G[3][3] = {{0.0}}, diva = 0.0;
        const double va[3] = {vx[a], vy[a], vz[a]}, aa[3] = {ax[a], ay[a], az[a]};
        for (int64_t k = nl.off[a]; k < nl.off[a + 1]; k++) {
            int64_t b = nl.ids[k];
            double d[3];
            double r = orc_dist(x, y, z, a, b, boxL, p->periodic, d);
            if (!(r < R * h[a])) continue;   /* the estimator uses W(h_a) only */
            double rhat[3] = {d[0] / r, d[1] / r, d[2] / r};
            double Fa = orc_F(r, h[a]);
            const double vb[3] = {vx[b], vy[b], vz[b]}, ab[3] = {ax[b], ay[b], az[b]};
            for (int i = 0; i < 3; i++) {
                for (int j = 0; j < 3; j++) G[i][j] += mass * (va[i] - vb[i]) * Fa * rhat[j];
                diva += mass * (aa[i] - ab[i]) * Fa * rhat[i];
            }
        }
        double rho = mass * pow(p->hfact / h[a], 3.0);
        double fac = -1.0 / (omega[a] * rho);
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) G[i][j] *= fac;   /* G[i][j] = d_j v^i */
        diva *= fac;
        double divv = G[0][0] + G[1][1] + G[2][2];
        double cx = G[2][1] - G[1][2], cy = G[0][2] - G[2][0], cz = G[1][0] - G[0][1];
        double tr = 0.0;
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) tr += G[i][j] * G[j][i];
        double ddiv = diva - tr;
        double den = divv * divv + (cx * cx + cy * cy + cz * cz);
        double xi = den > 0.0 ? divv * divv / den : 0.0;
        double A = xi * (ddiv < 0.0 ? -ddiv : 0.0);
        double cs = sqrt(p->gamma * (p->gamma - 1.0) * u[a]);
        double aloc = A > 0.0 ? p->alpha_av : 0.0;   /* c_s = 0: the limit of the ratio */
        if (cs > 0.0) {
            aloc = 10.0 * h[a] * h[a] * A / (cs * cs);
            if (aloc > p->alpha_av) aloc = p->alpha_av;
        }
        if (aloc < p->alpha_min) aloc = p->alpha_min;
        double q = cs > 0.0 ? dt * p->sigma_decay * cs / h[a] : 0.0;   /* dt / tau */
        double an = (alpha[a] + aloc * q) / (1.0 + q);
        alpha[a] = an > aloc ? an : aloc;
    }
    orc_nlist_free(&nl);
}

/* CFL time step (App. G, "Choice of the timestep"): min_a min(C_cour h_a / v_sig,a, C_force sqrt(h_a/|a_a|)). */
double orc_cfl(int64_t n, const orc_params *p, const double *h, const double *vsig,
               const double *ax, const double *ay, const double *az)
{
    double dt = INFINITY;
    for (int64_t a = 0; a < n; a++) {
        double t1 = p->c_cour * h[a] / vsig[a];
        double am = sqrt((ax[a] * ax[a] + ay[a] * ay[a]) + az[a] * az[a]);
        double t2 = am > 0.0 ? p->c_force * sqrt(h[a] / am) : INFINITY;
        double t = t1 < t2 ? t1 : t2;
        if (t < dt) dt = t;
    }
    return dt;
}

/* Periodic wrap of one coordinate into [lo, hi): x - L*floor((x-lo)/L); a result equal to hi
 * (rounding of a tiny negative offset) is set to lo. */
static double orc_wrap(double x, double lo, double hi)
{
    double L = hi - lo;
    double w = x - L * floor((x - lo) / L);
    if (w >= hi) w = lo;
    if (w < lo) w = lo;
    return w;
}

/* ====================================================================================== */
/* One kick-drift-kick step (App. G, "Leapfrog integration"):                                */
/*   v^{n+1/2} = v^n + dt/2 a^n;  r^{n+1} = r^n + dt v^{n+1/2} (wrapped);  v* = v^{n+1/2} + dt/2 a^n */
/*   u is advanced the same way with du/dt (reading);                                           */
/*   h, rho, Omega from Alg. F at r^{n+1};  a^{n+1}, du^{n+1} from (r^{n+1}, v*, u*);             */
/*   v^{n+1} = v* + dt/2 (a^{n+1} - a^n), likewise u.                                            */
/* State arrays are updated in place (original particle order).  Returns the CFL time step for  */
/* the next step, or a negative value if the h iteration failed.  dv_ratio (optional) receives   */
/* max_i |dv_i| / sqrt(<|v|^2>) for the correction dv_i = dt/2 (a^{n+1}_i - a^n_i) (Eq. deltavi;   */
/* reading of Eq. cvleapfrog, whose printed ratio is always >= 1).                              */
/* ====================================================================================== */
/* One step with the extensions of App. G: when alpha is non-NULL and p->av_switch, alpha_a is   */
/* updated (orc_alpha_update) after the h iteration and used by the forces; when p->eps_v > 0,    */
/* the corrector is re-run while Eq. cvleapfrog fails (reading below), at most p->max_corr passes, */
/* and *lambda (the CFL multiplier, NULL: none) is halved in a step whose first pass failed, else   */
/* relaxed by lambda <- (1 + lambda_stiff lambda)/(1 + lambda_stiff) ("CFL multiplier"); the      */
/* returned time step is lambda times the CFL step.  Reading of Eq. cvleapfrog (as printed its ratio is always >= 1): pass k compares */
/* max_i |v_i^(k) - w_i^(k)| = dt/2 |a_i^(k) - a_i^(k-1)| (a^(0) = a^n), w^(k) the velocity the     */
/* forces of pass k used (v* for k = 1, where the difference is Eq. deltavi; v^(k-1) afterwards,   */
/* the paper's "v* <- v^{n+1}"), with                                                              */
/* sqrt(<|v^(k)|^2>) and fails at >= eps_v (never when nothing moves).  Each pass restarts the     */
/* correction from v* and u*: v^(k) = v* + dt/2 (a^(k) - a^n).  *passes: corrector passes used.     */
double orc_step_ext(int64_t n, double mass, const orc_params *p, double dt,
                    double *x, double *y, double *z, double *vx, double *vy, double *vz, double *u, double *h,
                    double *ax, double *ay, double *az, double *du, double *rho, double *omega, double *vsig,
                    double *alpha, double *lambda, int method, int *iters, double *dv_ratio, int *passes)
{
    size_t sz = (size_t)(n > 0 ? n : 1) * sizeof(double);
    double *a0x = (double *)malloc(sz), *a0y = (double *)malloc(sz), *a0z = (double *)malloc(sz),
           *du0 = (double *)malloc(sz), *vsx = (double *)malloc(sz), *vsy = (double *)malloc(sz),
           *vsz = (double *)malloc(sz), *us = (double *)malloc(sz), *apx = (double *)malloc(sz),
           *apy = (double *)malloc(sz), *apz = (double *)malloc(sz);
    for (int64_t a = 0; a < n; a++) {
        a0x[a] = ax[a]; a0y[a] = ay[a]; a0z[a] = az[a]; du0[a] = du[a];
        apx[a] = ax[a]; apy[a] = ay[a]; apz[a] = az[a];
        double hvx = vx[a] + 0.5 * dt * ax[a], hvy = vy[a] + 0.5 * dt * ay[a], hvz = vz[a] + 0.5 * dt * az[a];
        double hu = u[a] + 0.5 * dt * du[a];
        x[a] = orc_wrap(x[a] + dt * hvx, p->lo[0], p->hi[0]);
        y[a] = orc_wrap(y[a] + dt * hvy, p->lo[1], p->hi[1]);
        z[a] = orc_wrap(z[a] + dt * hvz, p->lo[2], p->hi[2]);
        vx[a] = hvx + 0.5 * dt * ax[a];
        vy[a] = hvy + 0.5 * dt * ay[a];
        vz[a] = hvz + 0.5 * dt * az[a];
        u[a] = hu + 0.5 * dt * du[a];
        vsx[a] = vx[a]; vsy[a] = vy[a]; vsz[a] = vz[a]; us[a] = u[a];   /* v*, u* */
    }
    int outer = 0;
    int it = orc_density_algF(n, mass, p, x, y, z, h, rho, omega, method, &outer);
    if (iters) *iters = it;
    if (it < 0) {
        free(a0x); free(a0y); free(a0z); free(du0); free(vsx); free(vsy); free(vsz); free(us);
        free(apx); free(apy); free(apz);
        return -1.0;
    }
    const double *al = (p->av_switch && alpha) ? alpha : NULL;
    if (al) orc_alpha_update(n, mass, p, x, y, z, vx, vy, vz, a0x, a0y, a0z, u, h, omega, dt, method, alpha);
    double ratio = 0.0;
    int k = 0, failed = 0;
    for (;;) {
        k++;
        orc_forces_alpha(n, mass, p, x, y, z, vx, vy, vz, u, h, omega, al, method, ax, ay, az, du, vsig);
        double errmax = 0.0, v2 = 0.0;
        for (int64_t a = 0; a < n; a++) {
            /* v^(k) - w^(k) = dt/2 (a^(k) - a^(k-1)), a^(0) = a^n: both start from v* */
            double ex = 0.5 * dt * (ax[a] - apx[a]), ey = 0.5 * dt * (ay[a] - apy[a]),
                   ez = 0.5 * dt * (az[a] - apz[a]);
            double e = sqrt((ex * ex + ey * ey) + ez * ez);
            if (e > errmax) errmax = e;
            apx[a] = ax[a]; apy[a] = ay[a]; apz[a] = az[a];
            vx[a] = vsx[a] + 0.5 * dt * (ax[a] - a0x[a]);
            vy[a] = vsy[a] + 0.5 * dt * (ay[a] - a0y[a]);
            vz[a] = vsz[a] + 0.5 * dt * (az[a] - a0z[a]);
            u[a] = us[a] + 0.5 * dt * (du[a] - du0[a]);
            v2 += (vx[a] * vx[a] + vy[a] * vy[a]) + vz[a] * vz[a];
        }
        ratio = (v2 > 0.0) ? errmax / sqrt(v2 / (double)n) : 0.0;
        int fails = p->eps_v > 0.0 && !(ratio < p->eps_v);
        if (k == 1) {
            if (dv_ratio) *dv_ratio = ratio;
            failed = fails;
        }
        if (!fails || k >= p->max_corr) break;
    }
    if (passes) *passes = k;
    if (lambda) {
        if (failed) *lambda *= 0.5;
        else *lambda = (1.0 + p->lambda_stiff * *lambda) / (1.0 + p->lambda_stiff);
    }
    free(a0x); free(a0y); free(a0z); free(du0); free(vsx); free(vsy); free(vsz); free(us);
    free(apx); free(apy); free(apz);
    return (lambda ? *lambda : 1.0) * orc_cfl(n, p, h, vsig, ax, ay, az);
}

double orc_step(int64_t n, double mass, const orc_params *p, double dt,
                double *x, double *y, double *z, double *vx, double *vy, double *vz, double *u, double *h,
                double *ax, double *ay, double *az, double *du, double *rho, double *omega, double *vsig,
                int method, int *iters, double *dv_ratio)
{
    orc_params q = *p;
    q.av_switch = 0;
    q.eps_v = 0.0;
    return orc_step_ext(n, mass, &q, dt, x, y, z, vx, vy, vz, u, h, ax, ay, az, du, rho, omega, vsig, NULL, NULL,
                        method, iters, dv_ratio, NULL);
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ====================================================================================== */
/* Sampled evaluation for large inputs: the same definitions, for a list of particles only.   */
/* Candidates are found by brute force over all n; smoothing lengths are the roots of the      */
/* density equation (orc_density_root), Omega follows Eq. sphomega at those roots, and the      */
/* derivatives follow orc_forces term by term.                                                  */
/* ====================================================================================== */

/* Brute-force candidate list of particle a: every b != a within radius rad (nearest image). */
static int64_t orc_candidates(int64_t n, const double *x, const double *y, const double *z, int64_t a, double rad,
                              const double *boxL, int periodic, int64_t **out)
{
    int64_t cap = 256, k = 0;
    int64_t *l = (int64_t *)malloc((size_t)cap * sizeof(int64_t));
    for (int64_t b = 0; b < n; b++) {
        if (b == a) continue;
        double d[3];
        double r = orc_dist(x, y, z, a, b, boxL, periodic, d);
        if (r < rad) {
            if (k == cap) { cap *= 2; l = (int64_t *)realloc(l, (size_t)cap * sizeof(int64_t)); }
            l[k++] = b;
        }
    }
    *out = l;
    return k;
}

/* Root h (bisection of phi as in orc_density_root) and Omega of one particle from its candidate list. */
static void orc_one_root(int64_t a, const int64_t *cand, int64_t nc, const double *x, const double *y, const double *z,
                         double mass, double hfact, double h_hi, const double *boxL, int periodic,
                         double *h_out, double *om_out)
{
    orc_nlist one;
    int64_t *off = (int64_t *)malloc((size_t)(a + 2) * sizeof(int64_t));
    int32_t *ids = (int32_t *)malloc((size_t)(nc > 0 ? nc : 1) * sizeof(int32_t));
    for (int64_t i = 0; i <= a; i++) off[i] = 0;
    off[a + 1] = nc;
    for (int64_t k = 0; k < nc; k++) ids[k] = (int32_t)cand[k];
    one.n = a + 1; one.off = off; one.ids = ids;
    double hl = 0.0, hh = h_hi;
    for (int it = 0; it < 200; it++) {
        double hm = 0.5 * (hl + hh);
        if (hm <= hl || hm >= hh) break;
        if (hl > 0.0 && (hh - hl) <= 1e-16 * hh) break;
        if (orc_phi(a, hm, &one, x, y, z, boxL, periodic, hfact) > 0.0) hh = hm;
        else hl = hm;
    }
    double h = 0.5 * (hl + hh);
    if (!(orc_phi(a, h_hi, &one, x, y, z, boxL, periodic, hfact) > 0.0)) h = NAN;
    double rs, ds;
    orc_rho_sums(a, h, mass, &one, x, y, z, boxL, periodic, &rs, &ds);
    double rho_h = mass * pow(hfact / h, 3.0);
    *h_out = h;
    *om_out = 1.0 + h / (3.0 * rho_h) * ds;
    free(off); free(ids);
}

/* For m sampled particles idx[]: root h, Omega, and (ax, ay, az, du, vsig) from the definitions.
 * h_hi must exceed every smoothing length involved.  Returns the number of particles whose root
 * could not be bracketed (0 on success). */
int64_t orc_subset_forces(int64_t n, double mass, const orc_params *p, const double *x, const double *y,
                          const double *z, const double *vx, const double *vy, const double *vz, const double *u,
                          double h_hi, int64_t m, const int64_t *idx, double *h_o, double *om_o,
                          double *ax, double *ay, double *az, double *du, double *vs_o)
{
    double boxL[3] = {p->hi[0] - p->lo[0], p->hi[1] - p->lo[1], p->hi[2] - p->lo[2]};
    int64_t bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : bad)
    for (int64_t s = 0; s < m; s++) {
        int64_t a = idx[s];
        int64_t *cand;
        double R = orc_kernel_R(orc_kind);
        int64_t nc = orc_candidates(n, x, y, z, a, R * h_hi, boxL, p->periodic, &cand);
        double ha, oma;
        orc_one_root(a, cand, nc, x, y, z, mass, p->hfact, h_hi, boxL, p->periodic, &ha, &oma);
        double rho_a = mass * pow(p->hfact / ha, 3.0);
        double P_a = (p->gamma - 1.0) * rho_a * u[a];
        double c_a = sqrt(p->gamma * P_a / rho_a);
        double acc[3] = {0.0, 0.0, 0.0}, dua = 0.0, vs = p->alpha_av * c_a;
        if (!(ha == ha)) bad++;
        for (int64_t k = 0; k < nc; k++) {
            int64_t b = cand[k];
            int64_t *cb;
            int64_t nb = orc_candidates(n, x, y, z, b, R * h_hi, boxL, p->periodic, &cb);
            double hb, omb;
            orc_one_root(b, cb, nb, x, y, z, mass, p->hfact, h_hi, boxL, p->periodic, &hb, &omb);
            free(cb);
            if (!(hb == hb)) { bad++; continue; }
            double d[3];
            double r = orc_dist(x, y, z, a, b, boxL, p->periodic, d);
            double hm = ha > hb ? ha : hb;
            if (!(r < R * hm)) continue;
            double rho_b = mass * pow(p->hfact / hb, 3.0);
            double P_b = (p->gamma - 1.0) * rho_b * u[b];
            double c_b = sqrt(p->gamma * P_b / rho_b);
            double rhat[3] = {d[0] / r, d[1] / r, d[2] / r};
            double vdotr = (vx[a] - vx[b]) * rhat[0] + (vy[a] - vy[b]) * rhat[1] + (vz[a] - vz[b]) * rhat[2];
            double Fa = orc_F(r, ha), Fb = orc_F(r, hb);
            double qa = 0.0, qb = 0.0;
            if (vdotr < 0.0) {
                qa = -0.5 * rho_a * (p->alpha_av * c_a + p->beta_av * fabs(vdotr)) * vdotr;
                qb = -0.5 * rho_b * (p->alpha_av * c_b + p->beta_av * fabs(vdotr)) * vdotr;
            }
            double Aa = (P_a + qa) / (rho_a * rho_a * oma);
            double Ab = (P_b + qb) / (rho_b * rho_b * omb);
            double sc = mass * (Aa * Fa + Ab * Fb);
            for (int c = 0; c < 3; c++) acc[c] -= sc * rhat[c];
            dua += mass * Aa * vdotr * Fa;
            if (p->alpha_u != 0.0) {
                double vsu = sqrt(fabs(P_a - P_b) / (0.5 * (rho_a + rho_b)));
                dua += mass * p->alpha_u * vsu * (u[a] - u[b]) * 0.5 * (Fa / (oma * rho_a) + Fb / (omb * rho_b));
            }
            double vsdt = p->alpha_av * c_a + p->beta_av * (vdotr < 0.0 ? -vdotr : 0.0);
            if (vsdt > vs) vs = vsdt;
        }
        free(cand);
        h_o[s] = ha; om_o[s] = oma;
        ax[s] = acc[0]; ay[s] = acc[1]; az[s] = acc[2]; du[s] = dua; vs_o[s] = vs;
    }
    return bad;
}

/* Neighbour set (definition of orc_neighbours) of m sampled particles; off[m+1], ids sized by the
 * caller from a first call with ids == NULL (returns the total). */
int64_t orc_subset_neighbours(int64_t n, const double *x, const double *y, const double *z, const double *hc,
                              double s, const double *lo, const double *hi, int periodic, int64_t m,
                              const int64_t *idx, int64_t *off, int32_t *ids)
{
    double boxL[3] = {hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]};
    int64_t tot = 0;
    if (off) off[0] = 0;
    for (int64_t k = 0; k < m; k++) {
        int64_t a = idx[k];
        for (int64_t b = 0; b < n; b++)
            if (b != a && orc_pair_in(x, y, z, hc, a, b, s, boxL, periodic)) {
                if (ids) ids[tot] = (int32_t)b;
                tot++;
            }
        if (off) off[k + 1] = tot;
    }
    return tot;
}
