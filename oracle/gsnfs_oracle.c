/*
 * gsnfs_oracle.c -- plain, slow, FP64 CPU oracle of the GS-NFS per-frame codec.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link,
 * call or execute this file: only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark use it.  It shares no code, header, table
 * or constant generator with the CUDA library; the bitstream layout is
 * restated here from the written format description.
 *
 * Every function follows a passage of the paper (arxiv 2606.05650) and is
 * written as the plain definition, not as a copy of the paper's GPU listings:
 *   - voxelisation and cluster averaging          : Sec. 2.1, Sec. 2.2
 *   - Morton code                                  : Sec. 2.2 ("Morton Codes")
 *   - octree occupancy stream                      : Sec. 2.1 (recursive
 *     level-order traversal), header of Algorithm 1
 *   - octree decoding                              : Sec. 2.3, Algorithms 2-3
 *   - RAHT forward / inverse                       : Sec. 3.1, Eq. 1, App. D
 *   - P-RAHT schedule (used only to cross-check)   : Sec. 3.2, Algorithm 4
 *   - dead-zone / uniform quantiser                : Sec. 3.4
 *   - block RLGR                                   : Sec. 3.4, App. H (Table A.5)
 *   - occupancy entropy stage (own rANS, the paper
 *     uses a closed library ANS)                    : Sec. 2.2 last paragraph
 *
 * Floating point: FP64 throughout; no FMA contraction (build with
 * -ffp-contract=off) so that the voxel-grid arithmetic is one IEEE operation
 * per step and therefore reproducible bit for bit.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_CAPACITY (-2)
#define ORC_ERR_CORRUPT (-3)
#define ORC_ERR_NOMEM (-6)

/* ------------------------------------------------------------------------ */
/* Voxelisation (Sec. 2.1: cube grid of 2^J per axis over the bounding box;
 * Sec. 2.2: one thread per Gaussian computes its voxel coordinates).
 * Reading of the paper (it does not fix the arithmetic):
 *   lo_a  = min_i p_ia, hi_a = max_i p_ia         (exact)
 *   ext   = max_a (hi_a - lo_a) in FP64, 1 if it is 0   (one cube, isotropic)
 *   s     = 2^J / ext                              (one IEEE division)
 *   v_ia  = min(2^J - 1, floor(((double)p_ia - lo_a) * s))
 * Decoded position = voxel centre lo_a + (v + 0.5) * (ext / 2^J).          */
/* ------------------------------------------------------------------------ */
int orc_bbox(const float *pos, int64_t n, double lo[3], double *ext)
{
    if (n <= 0) {
        lo[0] = lo[1] = lo[2] = 0.0;
        *ext = 1.0;
        return ORC_OK;
    }
    double hi[3];
    for (int a = 0; a < 3; ++a) lo[a] = hi[a] = (double)pos[a];
    for (int64_t i = 1; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            double p = (double)pos[3 * i + a];
            if (p < lo[a]) lo[a] = p;
            if (p > hi[a]) hi[a] = p;
        }
    double e = 0.0;
    for (int a = 0; a < 3; ++a) {
        double d = hi[a] - lo[a];
        if (d > e) e = d;
    }
    *ext = (e > 0.0) ? e : 1.0;
    return ORC_OK;
}

void orc_voxel_coords(const float *pos, int64_t n, int J, const double lo[3], double ext,
                      uint32_t *vox)
{
    const double cells = ldexp(1.0, J);
    const double s = cells / ext;
    const uint64_t vmax = ((uint64_t)1 << J) - 1;
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            double t = (double)pos[3 * i + a] - lo[a];
            double u = floor(t * s);
            uint64_t v = (u <= 0.0) ? 0 : (uint64_t)u;
            if (v > vmax) v = vmax;
            vox[3 * i + a] = (uint32_t)v;
        }
}

/* Morton code (Sec. 2.2): bit string z_{J-1} y_{J-1} x_{J-1} ... z_0 y_0 x_0,
 * i.e. bit 3b is x_b, bit 3b+1 is y_b, bit 3b+2 is z_b; higher bits zero.   */
uint64_t orc_morton(uint32_t x, uint32_t y, uint32_t z, int J)
{
    uint64_t m = 0;
    for (int b = 0; b < J; ++b) {
        m |= (uint64_t)((x >> b) & 1u) << (3 * b);
        m |= (uint64_t)((y >> b) & 1u) << (3 * b + 1);
        m |= (uint64_t)((z >> b) & 1u) << (3 * b + 2);
    }
    return m;
}

void orc_morton_codes(const uint32_t *vox, int64_t n, int J, uint64_t *codes)
{
    for (int64_t i = 0; i < n; ++i) codes[i] = orc_morton(vox[3 * i], vox[3 * i + 1], vox[3 * i + 2], J);
}

void orc_morton_decode(uint64_t m, int J, uint32_t *x, uint32_t *y, uint32_t *z)
{
    uint32_t a = 0, b2 = 0, c = 0;
    for (int b = 0; b < J; ++b) {
        a |= (uint32_t)((m >> (3 * b)) & 1u) << b;
        b2 |= (uint32_t)((m >> (3 * b + 1)) & 1u) << b;
        c |= (uint32_t)((m >> (3 * b + 2)) & 1u) << b;
    }
    *x = a;
    *y = b2;
    *z = c;
}

void orc_voxel_centres(const uint64_t *codes, int64_t nv, int J, const double lo[3], double ext,
                       float *pos)
{
    const double cell = ext / ldexp(1.0, J);
    for (int64_t i = 0; i < nv; ++i) {
        uint32_t v[3];
        orc_morton_decode(codes[i], J, &v[0], &v[1], &v[2]);
        for (int a = 0; a < 3; ++a) {
            double off = ((double)v[a] + 0.5) * cell;
            pos[3 * i + a] = (float)(lo[a] + off);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Cluster averaging (Sec. 2.1 / 2.2): Gaussians sharing a voxel are replaced
 * by one whose attributes are the arithmetic mean of theirs.  The voxel set
 * is the set of distinct Morton codes in ascending order.  The mean is taken
 * in FP64 over the Gaussians in increasing input index.                     */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint64_t code;
    int64_t idx;
} orc_pair;

static int cmp_pair(const void *pa, const void *pb)
{
    const orc_pair *a = (const orc_pair *)pa, *b = (const orc_pair *)pb;
    if (a->code != b->code) return a->code < b->code ? -1 : 1;
    if (a->idx != b->idx) return a->idx < b->idx ? -1 : 1;
    return 0;
}

int64_t orc_merge(const uint64_t *codes, const float *attr, int64_t n, int C, uint64_t *out_codes,
                  double *out_attr, int64_t *out_counts)
{
    if (n <= 0) return 0;
    orc_pair *p = (orc_pair *)malloc(sizeof(orc_pair) * (size_t)n);
    if (!p) return ORC_ERR_NOMEM;
    for (int64_t i = 0; i < n; ++i) {
        p[i].code = codes[i];
        p[i].idx = i;
    }
    qsort(p, (size_t)n, sizeof(orc_pair), cmp_pair);
    int64_t nv = 0;
    int64_t i = 0;
    while (i < n) {
        int64_t j = i;
        while (j < n && p[j].code == p[i].code) ++j;
        out_codes[nv] = p[i].code;
        if (out_counts) out_counts[nv] = j - i;
        for (int c = 0; c < C; ++c) {
            double s = 0.0;
            for (int64_t k = i; k < j; ++k) s += (double)attr[(size_t)p[k].idx * C + c];
            out_attr[(size_t)nv * C + c] = s / (double)(j - i);
        }
        ++nv;
        i = j;
    }
    free(p);
    return nv;
}

/* ------------------------------------------------------------------------ */
/* Octree occupancy stream (Sec. 2.1 "Recursive Octree Encoding"): a single
 * level-order traversal from the root; each internal node emits one byte
 * whose bit i is set iff child i is occupied; children are visited in the
 * order 0..7.  Child index of a voxel at depth d is the bit triple
 * (z_b, y_b, x_b) with b = J-1-d, i = 4 z_b + 2 y_b + x_b (the Morton digit).
 * The traversal partitions the voxel coordinates top-down; it never sorts
 * by Morton code.  level_sizes[d] = number of occupied nodes at depth d
 * (header of Algorithm 1).  Returns the number of occupancy bytes.          */
/* ------------------------------------------------------------------------ */
int64_t orc_octree_encode(const uint32_t *vox, int64_t nv, int J, uint8_t *occ,
                          uint32_t *level_sizes)
{
    for (int d = 0; d <= J; ++d) level_sizes[d] = 0;
    if (nv <= 0) return 0;
    /* current level: nodes as [start,end) ranges into perm */
    int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)nv);
    int64_t *tmp = (int64_t *)malloc(sizeof(int64_t) * (size_t)nv);
    int64_t *ranges = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nv + 1) * 2);
    int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nv + 1) * 2);
    if (!perm || !tmp || !ranges || !next) {
        free(perm); free(tmp); free(ranges); free(next);
        return ORC_ERR_NOMEM;
    }
    for (int64_t i = 0; i < nv; ++i) perm[i] = i;
    int64_t nnodes = 1;
    ranges[0] = 0;
    ranges[1] = nv;
    int64_t nbytes = 0;
    for (int d = 0; d < J; ++d) {
        level_sizes[d] = (uint32_t)nnodes;
        const int b = J - 1 - d;
        int64_t nnext = 0;
        for (int64_t k = 0; k < nnodes; ++k) {
            const int64_t s = ranges[2 * k], e = ranges[2 * k + 1];
            int64_t cnt[8] = {0};
            for (int64_t t = s; t < e; ++t) {
                const uint32_t *v = vox + 3 * perm[t];
                int ci = (int)(((v[2] >> b) & 1u) << 2 | ((v[1] >> b) & 1u) << 1 | ((v[0] >> b) & 1u));
                cnt[ci]++;
            }
            uint8_t byte = 0;
            int64_t start[8];
            int64_t acc = s;
            for (int ci = 0; ci < 8; ++ci) {
                start[ci] = acc;
                acc += cnt[ci];
                if (cnt[ci]) byte |= (uint8_t)(1u << ci);
            }
            occ[nbytes++] = byte;
            int64_t fill[8];
            memcpy(fill, start, sizeof(fill));
            for (int64_t t = s; t < e; ++t) {
                const uint32_t *v = vox + 3 * perm[t];
                int ci = (int)(((v[2] >> b) & 1u) << 2 | ((v[1] >> b) & 1u) << 1 | ((v[0] >> b) & 1u));
                tmp[fill[ci]++] = perm[t];
            }
            for (int ci = 0; ci < 8; ++ci)
                if (cnt[ci]) {
                    next[2 * nnext] = start[ci];
                    next[2 * nnext + 1] = start[ci] + cnt[ci];
                    ++nnext;
                }
        }
        memcpy(perm, tmp, sizeof(int64_t) * (size_t)nv);
        int64_t *sw = ranges;
        ranges = next;
        next = sw;
        nnodes = nnext;
    }
    level_sizes[J] = (uint32_t)nnodes;
    free(perm); free(tmp); free(ranges); free(next);
    return nbytes;
}

/* Octree decoding (Sec. 2.3, Algorithms 2 and 3): start from the implicit
 * root code 0; per depth read |L_d| bytes, and for each parent in order emit
 * (parent << 3) + i for every set bit i.  Sizes are checked against the
 * header.  Returns |L_J| or a negative error.                              */
int64_t orc_octree_decode(const uint8_t *occ, int64_t n_occ, int J, const uint32_t *level_sizes,
                          uint64_t *leaves, int64_t cap)
{
    if (level_sizes[0] == 0) {
        for (int d = 0; d <= J; ++d)
            if (level_sizes[d] != 0) return ORC_ERR_CORRUPT;
        return n_occ == 0 ? 0 : ORC_ERR_CORRUPT;
    }
    if (level_sizes[0] != 1) return ORC_ERR_CORRUPT;
    int64_t maxl = 1;
    for (int d = 0; d <= J; ++d)
        if ((int64_t)level_sizes[d] > maxl) maxl = level_sizes[d];
    uint64_t *cur = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)maxl);
    uint64_t *nxt = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)maxl);
    if (!cur || !nxt) {
        free(cur); free(nxt);
        return ORC_ERR_NOMEM;
    }
    int64_t ncur = 1;
    cur[0] = 0;
    int64_t pos = 0;
    for (int d = 0; d < J; ++d) {
        if ((int64_t)level_sizes[d] != ncur || pos + ncur > n_occ) {
            free(cur); free(nxt);
            return ORC_ERR_CORRUPT;
        }
        int64_t nn = 0;
        for (int64_t p = 0; p < ncur; ++p) {
            uint8_t byte = occ[pos + p];
            if (byte == 0) {
                free(cur); free(nxt);
                return ORC_ERR_CORRUPT;
            }
            for (int i = 0; i < 8; ++i)
                if (byte & (1u << i)) {
                    if (nn >= (int64_t)level_sizes[d + 1]) {
                        free(cur); free(nxt);
                        return ORC_ERR_CORRUPT;
                    }
                    nxt[nn++] = (cur[p] << 3) + (uint64_t)i;
                }
        }
        pos += ncur;
        if (nn != (int64_t)level_sizes[d + 1]) {
            free(cur); free(nxt);
            return ORC_ERR_CORRUPT;
        }
        uint64_t *sw = cur;
        cur = nxt;
        nxt = sw;
        ncur = nn;
    }
    if (pos != n_occ || ncur > cap) {
        free(cur); free(nxt);
        return pos != n_occ ? ORC_ERR_CORRUPT : ORC_ERR_CAPACITY;
    }
    memcpy(leaves, cur, sizeof(uint64_t) * (size_t)ncur);
    free(cur); free(nxt);
    return ncur;
}

/* ------------------------------------------------------------------------ */
/* RAHT (Sec. 3.1, Eq. 1).  Binary tree: node at binary level l (0 = voxel)
 * is the set of voxels sharing M >> l; its two children at level l-1 are
 * split by bit l-1 of the Morton code (x, then y, then z, repeating).  When
 * both children are occupied, Eq. 1 maps their low-pass values (a_l, a_r)
 * with weights (w_l, w_r) = voxel counts to
 *   a0 = ( sqrt(w_l) a_l + sqrt(w_r) a_r) / sqrt(w_l + w_r)   (low  pass)
 *   a1 = (-sqrt(w_r) a_l + sqrt(w_l) a_r) / sqrt(w_l + w_r)   (high pass)
 * the low pass travels up, the high pass is stored at the right child.  A
 * node with one occupied child passes the value up unchanged.  Storage is
 * in place over the Morton-sorted voxel index (App. D): the low pass of a
 * node lives at its first voxel, the high pass of a split at the first
 * voxel of the right child, the DC ends at index 0.  The recursion runs
 * over all 3J binary levels so the two halves of the root also merge.
 * Coefficients are computed as a = sqrt(w_l/(w_l+w_r)), b = sqrt(w_r/(..)),
 * which is Eq. 1 rewritten (App. D).                                      */
/* ------------------------------------------------------------------------ */
typedef struct {
    const uint64_t *M;
    int C;
    double *Y;
    double *tmp;
} raht_ctx;

/* returns index of the first voxel in [lo,hi) whose bit (l-1) is set */
static int64_t raht_split(const uint64_t *M, int64_t lo, int64_t hi, int l)
{
    int64_t s = lo;
    while (s < hi && ((M[s] >> (l - 1)) & 1u) == 0) ++s;
    return s;
}

static void raht_fwd_rec(raht_ctx *cx, int64_t lo, int64_t hi, int l)
{
    if (l == 0 || hi - lo <= 1) return; /* single voxel: value already in place */
    int64_t s = raht_split(cx->M, lo, hi, l);
    if (s > lo) raht_fwd_rec(cx, lo, s, l - 1);
    if (s < hi) raht_fwd_rec(cx, s, hi, l - 1);
    if (s > lo && s < hi) {
        double wl = (double)(s - lo), wr = (double)(hi - s);
        double a = sqrt(wl / (wl + wr)), b = sqrt(wr / (wl + wr));
        double *yl = cx->Y + (size_t)lo * cx->C, *yr = cx->Y + (size_t)s * cx->C;
        for (int c = 0; c < cx->C; ++c) {
            double l0 = yl[c], r0 = yr[c];
            yl[c] = a * l0 + b * r0;
            yr[c] = -b * l0 + a * r0;
        }
    }
}

static void raht_inv_rec(raht_ctx *cx, int64_t lo, int64_t hi, int l)
{
    if (l == 0 || hi - lo <= 1) return;
    int64_t s = raht_split(cx->M, lo, hi, l);
    if (s > lo && s < hi) {
        double wl = (double)(s - lo), wr = (double)(hi - s);
        double a = sqrt(wl / (wl + wr)), b = sqrt(wr / (wl + wr));
        double *yl = cx->Y + (size_t)lo * cx->C, *yr = cx->Y + (size_t)s * cx->C;
        for (int c = 0; c < cx->C; ++c) {
            double lo0 = yl[c], hi0 = yr[c];
            yl[c] = a * lo0 - b * hi0;
            yr[c] = b * lo0 + a * hi0;
        }
    }
    if (s > lo) raht_inv_rec(cx, lo, s, l - 1);
    if (s < hi) raht_inv_rec(cx, s, hi, l - 1);
}

void orc_raht_forward(const uint64_t *M, int64_t nv, int J, int C, const double *A, double *Y)
{
    memmove(Y, A, sizeof(double) * (size_t)nv * (size_t)C);
    raht_ctx cx = {M, C, Y, NULL};
    if (nv > 1) raht_fwd_rec(&cx, 0, nv, 3 * J);
}

void orc_raht_inverse(const uint64_t *M, int64_t nv, int J, int C, const double *Yin, double *A)
{
    memmove(A, Yin, sizeof(double) * (size_t)nv * (size_t)C);
    raht_ctx cx = {M, C, A, NULL};
    if (nv > 1) raht_inv_rec(&cx, 0, nv, 3 * J);
}

/* Level of detail (decoding to octree depth Jp <= J; Algorithm 2's shift read as
 * J - Jp): the nodes of depth Jp are the distinct codes >> 3(J - Jp); each
 * gets the centre of its cell at depth Jp and the FP64 mean of its voxels'
 * attributes.  Returns the node count.                                      */
int64_t orc_lod(const uint64_t *M, int64_t nv, int J, int Jp, int C, const double *A, const double lo[3],
                double ext, uint64_t *node_codes, float *node_pos, double *node_attr, int64_t *node_w)
{
    if (Jp < 0 || Jp > J) return ORC_ERR_ARG;
    const int sh = 3 * (J - Jp);
    int64_t k = -1;
    for (int64_t i = 0; i < nv; ++i) {
        const uint64_t m = (sh >= 64) ? 0 : (M[i] >> sh);
        if (k < 0 || m != node_codes[k]) {
            ++k;
            node_codes[k] = m;
            node_w[k] = 0;
            for (int c = 0; c < C; ++c) node_attr[(size_t)k * C + c] = 0.0;
        }
        node_w[k] += 1;
        for (int c = 0; c < C; ++c) node_attr[(size_t)k * C + c] += A[(size_t)i * C + c];
    }
    const int64_t n = k + 1;
    for (int64_t j = 0; j < n; ++j)
        for (int c = 0; c < C; ++c) node_attr[(size_t)j * C + c] /= (double)node_w[j];
    orc_voxel_centres(node_codes, n, Jp, lo, ext, node_pos);
    return n;
}

/* Low-pass coefficient of every node at binary level l (Eq. 1 applied up to
 * level l inside each node, by the recursion of orc_raht_forward): out[k]
 * for the k-th node in Morton order, w[k] its voxel count.  By induction on
 * Eq. (1) it equals sqrt(w) times the mean of the node's values.           */
int64_t orc_raht_lowpass(const uint64_t *M, int64_t nv, int J, int C, const double *A, int l, double *out,
                         int64_t *w)
{
    double *Y = (double *)malloc(sizeof(double) * (size_t)(nv ? nv : 1) * (size_t)(C ? C : 1));
    if (!Y) return ORC_ERR_NOMEM;
    memcpy(Y, A, sizeof(double) * (size_t)nv * (size_t)C);
    raht_ctx cx = {M, C, Y, NULL};
    int64_t n = 0;
    for (int64_t lo = 0; lo < nv;) {
        const uint64_t key = (l >= 64) ? 0 : (M[lo] >> l);
        int64_t hi = lo + 1;
        while (hi < nv && ((l >= 64) ? 0 : (M[hi] >> l)) == key) ++hi;
        raht_fwd_rec(&cx, lo, hi, l);
        for (int c = 0; c < C; ++c) out[(size_t)n * C + c] = Y[(size_t)lo * C + c];
        w[n] = hi - lo;
        ++n;
        lo = hi;
    }
    free(Y);
    (void)J;
    return n;
}

/* Per-voxel "node weight" of each stored coefficient: w0+w1 of the split that
 * produced the high pass at that index, N_v for the DC at index 0.  Used by
 * the parity tolerance (FP32 error of a weighted sum of w inputs).          */
static void raht_w_rec(const uint64_t *M, int64_t lo, int64_t hi, int l, int64_t *w)
{
    if (l == 0 || hi - lo <= 1) return;
    int64_t s = raht_split(M, lo, hi, l);
    if (s > lo && s < hi) w[s] = hi - lo;
    if (s > lo) raht_w_rec(M, lo, s, l - 1, w);
    if (s < hi) raht_w_rec(M, s, hi, l - 1, w);
}

void orc_raht_node_weights(const uint64_t *M, int64_t nv, int J, int64_t *w)
{
    for (int64_t i = 0; i < nv; ++i) w[i] = 1;
    if (nv > 0) w[0] = nv;
    if (nv > 1) raht_w_rec(M, 0, nv, 3 * J, w);
}

/* P-RAHT schedule (Sec. 3.2, Algorithm 4), as an independent restatement used
 * only by tests to check that the listing's level lists describe the same
 * butterflies as the recursive definition.  Level l runs 1..3J (the reading
 * taken where the transform listing stops at 3J-1).  Writes one record per
 * butterfly: (level, i0, i1, w0, w1).  Returns the count (N_v - 1).        */
int64_t orc_praht_schedule(const uint64_t *M, int64_t nv, int J, int32_t *level, int64_t *i0,
                           int64_t *i1, int64_t *w0, int64_t *w1)
{
    if (nv <= 1) return 0;
    int64_t *I = (int64_t *)malloc(sizeof(int64_t) * (size_t)nv);
    int64_t *In = (int64_t *)malloc(sizeof(int64_t) * (size_t)nv);
    uint8_t *F = (uint8_t *)malloc((size_t)nv);
    if (!I || !In || !F) {
        free(I); free(In); free(F);
        return ORC_ERR_NOMEM;
    }
    int64_t n = nv, cnt = 0;
    for (int64_t k = 0; k < nv; ++k) I[k] = k;
    for (int l = 1; l <= 3 * J; ++l) {
        /* mask 2^{3J} - 2^l: the bits at and above l must agree */
        uint64_t mask = (l >= 64) ? 0 : (~(uint64_t)0 << l);
        if (3 * J < 64) mask &= (((uint64_t)1 << (3 * J)) - 1);
        for (int64_t k = 0; k < n; ++k) {
            F[k] = 0;
            if (k + 1 < n) F[k] = ((M[I[k]] ^ M[I[k + 1]]) & mask) == 0;
        }
        for (int64_t k = 0; k + 1 < n; ++k)
            if (F[k]) {
                int64_t nx = (k + 2 < n) ? I[k + 2] : nv;
                level[cnt] = l;
                i0[cnt] = I[k];
                i1[cnt] = I[k + 1];
                w0[cnt] = I[k + 1] - I[k];
                w1[cnt] = nx - I[k + 1];
                ++cnt;
            }
        /* next active list keeps left siblings and singletons */
        int64_t m = 0;
        for (int64_t k = 0; k < n; ++k)
            if (!(k > 0 && F[k - 1])) In[m++] = I[k];
        memcpy(I, In, sizeof(int64_t) * (size_t)m);
        n = m;
    }
    free(I); free(In); free(F);
    return cnt;
}

/* ------------------------------------------------------------------------ */
/* Quantiser (Sec. 3.4): dead-zone uniform scalar quantiser per attribute
 * group,  q = sign(y) floor(|y| / step + tau),  reconstruction q * step.
 * tau = 1/2 is the plain mid-tread uniform quantiser; smaller tau widens the
 * dead zone.  Magnitudes are clamped to 2^30.                              */
/* ------------------------------------------------------------------------ */
void orc_quantize(const double *Y, int64_t nv, int C, const uint8_t *group, const double *steps,
                  double tau, int32_t *Q)
{
    for (int64_t i = 0; i < nv; ++i)
        for (int c = 0; c < C; ++c) {
            double y = Y[(size_t)i * C + c];
            double t = floor(fabs(y) / steps[group[c]] + tau);
            if (t > 1073741824.0) t = 1073741824.0;
            int32_t m = (int32_t)t;
            Q[(size_t)i * C + c] = (y < 0.0) ? -m : m;
        }
}

/* ------------------------------------------------------------------------ */
/* Block RLGR (Sec. 3.4; App. H): run-length coding of zeros plus adaptive
 * Golomb-Rice coding of magnitudes (Malvar, DCC 2006), each block coded
 * independently.  The paper gives no constants; the ones below are this
 * codec's and are restated from the format description:
 *   u = 2q (q >= 0), -2q-1 (q < 0);  k = K >> 4, kR = KR >> 4;
 *   start of block: K = 0, KR = 32.
 *   k == 0: GR(u, kR); K += 3 if u == 0 else K -= 3 (floor 0).
 *   k > 0 : 2^k zeros ahead -> bit 0, K += 4 (cap 240);
 *           else r < 2^k zeros then u != 0 -> bit 1, r in k bits,
 *           GR(u-1, kR), K -= 6 (floor 0);
 *           block ends inside the run -> bit 0 (decoder clamps).
 *   GR(v, k): p = v >> k; p < 24: p ones, a zero, k low bits of v;
 *            else 24 ones, 6-bit length n of v, n bits of v.
 *   after GR(v): p == 0 -> KR -= 2 (floor 0); p > 1 -> KR += p + 1 (cap 384)
 *   bits are written least-significant first into 32-bit words; a block is
 *   padded to a whole word.                                               */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint32_t *w;
    int64_t cap;    /* words */
    int64_t nbits;
    int overflow;
} bitw;

static void bw_put(bitw *b, uint64_t v, int n)
{
    for (int i = 0; i < n; ++i) {
        int64_t word = b->nbits >> 5;
        if (word >= b->cap) {
            b->overflow = 1;
            return;
        }
        if ((b->nbits & 31) == 0) b->w[word] = 0;
        if ((v >> i) & 1u) b->w[word] |= (uint32_t)1u << (b->nbits & 31);
        b->nbits++;
    }
}

static void gr_put(bitw *b, uint32_t v, int k, int *KR)
{
    uint32_t p = v >> k;
    if (p < 24) {
        for (uint32_t i = 0; i < p; ++i) bw_put(b, 1, 1);
        bw_put(b, 0, 1);
        bw_put(b, v, k);
    } else {
        int n = 0;
        while (n < 32 && (v >> n) != 0) ++n;
        for (int i = 0; i < 24; ++i) bw_put(b, 1, 1);
        bw_put(b, (uint64_t)n, 6);
        bw_put(b, v, n);
    }
    if (p == 0) {
        *KR -= 2;
        if (*KR < 0) *KR = 0;
    } else if (p > 1) {
        int64_t t = (int64_t)*KR + (int64_t)p + 1;
        *KR = (t > 384) ? 384 : (int)t;
    }
}

static uint32_t zigzag(int32_t q)
{
    return q >= 0 ? (uint32_t)q << 1 : ((uint32_t)(-(int64_t)q) << 1) - 1u;
}

static int32_t unzigzag(uint32_t u)
{
    return (u & 1u) ? (int32_t)(-(int64_t)((u >> 1) + 1)) : (int32_t)(u >> 1);
}

/* Encodes n values of q (with stride) into words; returns words used or -2. */
int64_t orc_rlgr_encode(const int32_t *q, int64_t n, int64_t stride, uint32_t *words, int64_t cap)
{
    bitw b = {words, cap, 0, 0};
    int K = 0, KR = 32;
    int64_t i = 0;
    while (i < n) {
        int k = K >> 4;
        if (k == 0) {
            uint32_t u = zigzag(q[i * stride]);
            gr_put(&b, u, KR >> 4, &KR);
            if (u == 0) {
                K += 3;
                if (K > 240) K = 240;
            } else {
                K -= 3;
                if (K < 0) K = 0;
            }
            ++i;
        } else {
            int64_t run = (int64_t)1 << k;
            int64_t r = 0;
            while (r < run && i + r < n && q[(i + r) * stride] == 0) ++r;
            if (r == run || i + r == n) {
                bw_put(&b, 0, 1);
                i += r;
                K += 4;
                if (K > 240) K = 240;
            } else {
                uint32_t u = zigzag(q[(i + r) * stride]);
                bw_put(&b, 1, 1);
                bw_put(&b, (uint64_t)r, k);
                gr_put(&b, u - 1u, KR >> 4, &KR);
                K -= 6;
                if (K < 0) K = 0;
                i += r + 1;
            }
        }
    }
    if (b.overflow) return ORC_ERR_CAPACITY;
    return (b.nbits + 31) >> 5;
}

typedef struct {
    const uint32_t *w;
    int64_t nwords;
    int64_t pos;
    int bad;
} bitr;

static uint32_t br_get(bitr *b, int n)
{
    uint32_t v = 0;
    for (int i = 0; i < n; ++i) {
        int64_t word = b->pos >> 5;
        if (word >= b->nwords) {
            b->bad = 1;
            return 0;
        }
        uint32_t bit = (b->w[word] >> (b->pos & 31)) & 1u;
        v |= bit << i;
        b->pos++;
    }
    return v;
}

static uint32_t gr_get(bitr *b, int k, int *KR)
{
    uint32_t p = 0;
    while (p < 24 && br_get(b, 1) == 1u) {
        ++p;
        if (b->bad) return 0;
    }
    uint32_t v;
    if (p < 24) {
        v = (p << k) | br_get(b, k);
    } else {
        int n = (int)br_get(b, 6);
        if (n > 32) {
            b->bad = 1;
            return 0;
        }
        v = br_get(b, n);
        p = v >> k;
    }
    if (p == 0) {
        *KR -= 2;
        if (*KR < 0) *KR = 0;
    } else if (p > 1) {
        int64_t t = (int64_t)*KR + (int64_t)p + 1;
        *KR = (t > 384) ? 384 : (int)t;
    }
    return v;
}

int orc_rlgr_decode(const uint32_t *words, int64_t nwords, int64_t n, int64_t stride, int32_t *q)
{
    bitr b = {words, nwords, 0, 0};
    int K = 0, KR = 32;
    int64_t i = 0;
    while (i < n) {
        int k = K >> 4;
        if (k == 0) {
            uint32_t u = gr_get(&b, KR >> 4, &KR);
            if (b.bad) return ORC_ERR_CORRUPT;
            q[i * stride] = unzigzag(u);
            if (u == 0) {
                K += 3;
                if (K > 240) K = 240;
            } else {
                K -= 3;
                if (K < 0) K = 0;
            }
            ++i;
        } else {
            uint32_t bit = br_get(&b, 1);
            if (b.bad) return ORC_ERR_CORRUPT;
            if (bit == 0) {
                int64_t run = (int64_t)1 << k;
                if (run > n - i) run = n - i;
                for (int64_t t = 0; t < run; ++t) q[(i + t) * stride] = 0;
                i += run;
                K += 4;
                if (K > 240) K = 240;
            } else {
                int64_t r = br_get(&b, k);
                uint32_t v = gr_get(&b, KR >> 4, &KR);
                if (b.bad || i + r >= n || v == 0xFFFFFFFFu) return ORC_ERR_CORRUPT;
                for (int64_t t = 0; t < r; ++t) q[(i + t) * stride] = 0;
                q[(i + r) * stride] = unzigzag(v + 1u);
                K -= 6;
                if (K < 0) K = 0;
                i += r + 1;
            }
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Occupancy entropy stage.  The paper codes the occupancy bytes with a
 * closed library ANS (Sec. 2.2, Sec. 5.1); this codec uses its own static
 * order-0 rANS (Duda 2013) with 32 interleaved states (Giesen 2014):
 *   probabilities scaled to M = 2^15: f_s = floor(cnt_s M / n), at least 1
 *   for a present symbol; the most frequent symbol (lowest value on ties)
 *   absorbs M - sum f.  32-bit states, L = 2^16, 16-bit renormalisation.
 *   Symbol j of a chunk is coded by state j mod 32; the encoder runs from the
 *   last symbol to the first and its 16-bit words are stored in the order the
 *   decoder reads them.  Chunk = 32 final states (u32) + words (u16), padded
 *   to 4 bytes.                                                           */
/* ------------------------------------------------------------------------ */
#define RANS_PROB_BITS 15
#define RANS_M (1u << RANS_PROB_BITS)
#define RANS_L (1u << 16)
#define RANS_LANES 32

void orc_rans_freqs(const uint8_t *in, int64_t n, uint16_t freq[256])
{
    int64_t cnt[256] = {0};
    for (int64_t i = 0; i < n; ++i) cnt[in[i]]++;
    int best = 0;
    for (int s = 1; s < 256; ++s)
        if (cnt[s] > cnt[best]) best = s;
    int64_t sum = 0;
    int64_t f[256];
    for (int s = 0; s < 256; ++s) {
        f[s] = 0;
        if (cnt[s] > 0) {
            f[s] = (int64_t)(((uint64_t)cnt[s] * RANS_M) / (uint64_t)n);
            if (f[s] == 0) f[s] = 1;
        }
        sum += f[s];
    }
    f[best] += (int64_t)RANS_M - sum;
    for (int s = 0; s < 256; ++s) freq[s] = (uint16_t)f[s];
}

/* Encodes one chunk; returns its byte size (multiple of 4). */
static int64_t rans_chunk_encode(const uint8_t *sym, int64_t n, const uint16_t *freq,
                                 const uint32_t *cum, uint8_t *out)
{
    uint32_t x[RANS_LANES];
    for (int l = 0; l < RANS_LANES; ++l) x[l] = RANS_L;
    uint16_t *stack = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)(n + 1));
    int64_t nw = 0;
    for (int64_t j = n - 1; j >= 0; --j) {
        int l = (int)(j % RANS_LANES);
        uint32_t f = freq[sym[j]], c = cum[sym[j]];
        uint64_t xmax = ((uint64_t)(RANS_L >> RANS_PROB_BITS) << 16) * f;
        if ((uint64_t)x[l] >= xmax) {
            stack[nw++] = (uint16_t)(x[l] & 0xFFFFu);
            x[l] >>= 16;
        }
        x[l] = ((x[l] / f) << RANS_PROB_BITS) + (x[l] % f) + c;
    }
    for (int l = 0; l < RANS_LANES; ++l) {
        out[4 * l + 0] = (uint8_t)(x[l]);
        out[4 * l + 1] = (uint8_t)(x[l] >> 8);
        out[4 * l + 2] = (uint8_t)(x[l] >> 16);
        out[4 * l + 3] = (uint8_t)(x[l] >> 24);
    }
    /* decoder reads the last emitted word first */
    for (int64_t t = 0; t < nw; ++t) {
        uint16_t w = stack[nw - 1 - t];
        out[128 + 2 * t] = (uint8_t)w;
        out[128 + 2 * t + 1] = (uint8_t)(w >> 8);
    }
    free(stack);
    int64_t bytes = 128 + 2 * nw;
    while (bytes & 3) out[bytes++] = 0;
    return bytes;
}

static int rans_chunk_decode(const uint8_t *in, int64_t nbytes, int64_t n, const uint16_t *freq,
                             const uint32_t *cum, const uint8_t *slot2sym, uint8_t *out)
{
    if (nbytes < 128) return ORC_ERR_CORRUPT;
    uint32_t x[RANS_LANES];
    for (int l = 0; l < RANS_LANES; ++l)
        x[l] = (uint32_t)in[4 * l] | (uint32_t)in[4 * l + 1] << 8 | (uint32_t)in[4 * l + 2] << 16 |
               (uint32_t)in[4 * l + 3] << 24;
    int64_t wp = 128;
    for (int64_t j = 0; j < n; ++j) {
        int l = (int)(j % RANS_LANES);
        uint32_t slot = x[l] & (RANS_M - 1);
        uint8_t s = slot2sym[slot];
        out[j] = s;
        x[l] = (uint32_t)freq[s] * (x[l] >> RANS_PROB_BITS) + slot - cum[s];
        if (x[l] < RANS_L) {
            if (wp + 2 > nbytes) return ORC_ERR_CORRUPT;
            x[l] = (x[l] << 16) | (uint32_t)in[wp] | (uint32_t)in[wp + 1] << 8;
            wp += 2;
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Little-endian helpers for the container                                  */
/* ------------------------------------------------------------------------ */
static void put32(uint8_t *p, uint32_t v)
{
    for (int i = 0; i < 4; ++i) p[i] = (uint8_t)(v >> (8 * i));
}
static void put64(uint8_t *p, uint64_t v)
{
    for (int i = 0; i < 8; ++i) p[i] = (uint8_t)(v >> (8 * i));
}
static void putf64(uint8_t *p, double d)
{
    uint64_t v;
    memcpy(&v, &d, 8);
    put64(p, v);
}
static uint32_t get32(const uint8_t *p)
{
    uint32_t v = 0;
    for (int i = 0; i < 4; ++i) v |= (uint32_t)p[i] << (8 * i);
    return v;
}
static uint64_t get64(const uint8_t *p)
{
    uint64_t v = 0;
    for (int i = 0; i < 8; ++i) v |= (uint64_t)p[i] << (8 * i);
    return v;
}
static double getf64(const uint8_t *p)
{
    uint64_t v = get64(p);
    double d;
    memcpy(&d, &v, 8);
    return d;
}

/* Occupancy section (8-byte aligned):
 *   u64 n_occ; u32 mode; u32 aux
 *   mode 0 (raw)      : aux = 0, n_occ bytes, zero padded to 8
 *   mode 2 (constant) : aux = the byte value
 *   mode 1 (rANS)     : aux = n_chunks; u32 chunk_syms; u32 0;
 *                       u16 freq[256]; u32 chunk_bytes[n_chunks];
 *                       (pad to 8); chunk payloads; pad to 8
 * rANS is used when it is strictly smaller than raw.                       */
int64_t orc_occ_section_encode(const uint8_t *occ, int64_t n, uint32_t chunk_syms, uint8_t *out,
                               int64_t cap)
{
    if (chunk_syms == 0 || (chunk_syms % RANS_LANES) != 0) return ORC_ERR_ARG;
    int distinct = 0, val = 0;
    int seen[256] = {0};
    for (int64_t i = 0; i < n; ++i)
        if (!seen[occ[i]]) {
            seen[occ[i]] = 1;
            distinct++;
            val = occ[i];
        }
    int64_t raw_bytes = 16 + ((n + 7) & ~(int64_t)7);
    if (n > 0 && distinct == 1) {
        if (cap < 16) return ORC_ERR_CAPACITY;
        put64(out, (uint64_t)n);
        put32(out + 8, 2);
        put32(out + 12, (uint32_t)val);
        return 16;
    }
    int64_t rans_total = -1;
    uint8_t *rbuf = NULL;
    if (n > 0) {
        uint16_t freq[256];
        uint32_t cum[256];
        orc_rans_freqs(occ, n, freq);
        uint32_t acc = 0;
        for (int s = 0; s < 256; ++s) {
            cum[s] = acc;
            acc += freq[s];
        }
        int64_t nch = (n + chunk_syms - 1) / chunk_syms;
        int64_t table = 16 + 8 + 512 + 4 * nch;
        table = (table + 7) & ~(int64_t)7;
        int64_t bound = table + nch * (128 + 2 * (int64_t)chunk_syms + 4) + 8;
        rbuf = (uint8_t *)calloc((size_t)bound, 1);
        if (!rbuf) return ORC_ERR_NOMEM;
        put64(rbuf, (uint64_t)n);
        put32(rbuf + 8, 1);
        put32(rbuf + 12, (uint32_t)nch);
        put32(rbuf + 16, chunk_syms);
        put32(rbuf + 20, 0);
        for (int s = 0; s < 256; ++s) {
            rbuf[24 + 2 * s] = (uint8_t)freq[s];
            rbuf[24 + 2 * s + 1] = (uint8_t)(freq[s] >> 8);
        }
        int64_t pos = table;
        for (int64_t c = 0; c < nch; ++c) {
            int64_t s0 = c * chunk_syms;
            int64_t len = (n - s0 < chunk_syms) ? n - s0 : chunk_syms;
            int64_t b = rans_chunk_encode(occ + s0, len, freq, cum, rbuf + pos);
            put32(rbuf + 24 + 512 + 4 * c, (uint32_t)b);
            pos += b;
        }
        pos = (pos + 7) & ~(int64_t)7;
        rans_total = pos;
    }
    if (rans_total > 0 && rans_total < raw_bytes) {
        if (cap < rans_total) {
            free(rbuf);
            return ORC_ERR_CAPACITY;
        }
        memcpy(out, rbuf, (size_t)rans_total);
        free(rbuf);
        return rans_total;
    }
    free(rbuf);
    if (cap < raw_bytes) return ORC_ERR_CAPACITY;
    memset(out, 0, (size_t)raw_bytes);
    put64(out, (uint64_t)n);
    put32(out + 8, 0);
    put32(out + 12, 0);
    memcpy(out + 16, occ, (size_t)n);
    return raw_bytes;
}

int64_t orc_occ_section_decode(const uint8_t *in, int64_t nbytes, uint8_t *occ, int64_t cap)
{
    if (nbytes < 16) return ORC_ERR_CORRUPT;
    int64_t n = (int64_t)get64(in);
    uint32_t mode = get32(in + 8), aux = get32(in + 12);
    if (n < 0 || n > cap) return ORC_ERR_CORRUPT;
    if (mode == 2) {
        if (aux > 255) return ORC_ERR_CORRUPT;
        memset(occ, (int)aux, (size_t)n);
        return n;
    }
    if (mode == 0) {
        if (16 + n > nbytes) return ORC_ERR_CORRUPT;
        memcpy(occ, in + 16, (size_t)n);
        return n;
    }
    if (mode != 1) return ORC_ERR_CORRUPT;
    int64_t nch = aux;
    uint32_t chunk_syms = get32(in + 16);
    if (chunk_syms == 0 || chunk_syms % RANS_LANES) return ORC_ERR_CORRUPT;
    if (nch != (n + chunk_syms - 1) / chunk_syms) return ORC_ERR_CORRUPT;
    int64_t table = ((16 + 8 + 512 + 4 * nch) + 7) & ~(int64_t)7;
    if (table > nbytes) return ORC_ERR_CORRUPT;
    uint16_t freq[256];
    uint32_t cum[256];
    uint32_t acc = 0;
    for (int s = 0; s < 256; ++s) {
        freq[s] = (uint16_t)(in[24 + 2 * s] | (in[24 + 2 * s + 1] << 8));
        cum[s] = acc;
        acc += freq[s];
    }
    if (acc != RANS_M) return ORC_ERR_CORRUPT;
    uint8_t *slot2sym = (uint8_t *)malloc(RANS_M);
    if (!slot2sym) return ORC_ERR_NOMEM;
    for (int s = 0; s < 256; ++s)
        for (uint32_t t = 0; t < freq[s]; ++t) slot2sym[cum[s] + t] = (uint8_t)s;
    int64_t pos = table;
    for (int64_t c = 0; c < nch; ++c) {
        int64_t b = get32(in + 24 + 512 + 4 * c);
        int64_t s0 = c * chunk_syms;
        int64_t len = (n - s0 < chunk_syms) ? n - s0 : chunk_syms;
        if (pos + b > nbytes || b < 128 || (b & 3)) {
            free(slot2sym);
            return ORC_ERR_CORRUPT;
        }
        int r = rans_chunk_decode(in + pos, b, len, freq, cum, slot2sym, occ + s0);
        if (r) {
            free(slot2sym);
            return r;
        }
        pos += b;
    }
    free(slot2sym);
    return n;
}

/* ------------------------------------------------------------------------ */
/* Frame container (all little endian; every section starts 8-aligned)
 *   header, 96 bytes:
 *     0 u32 magic 0x314E5347 ("GSN1")   4 u32 version 1
 *     8 u32 header_bytes               12 u32 J
 *    16 u32 C                          20 u32 G
 *    24 u64 N_v                        32 f64 lo[3]
 *    56 f64 ext                        64 f64 tau
 *    72 u64 occ_section_bytes          80 u64 attr_section_bytes
 *    88 u32 flags (0)                  92 u32 reserved (0)
 *   then u32 level_size[J+1], u8 group[C], pad to 8, f64 step[G].
 *   occupancy section (above).
 *   attribute section (absent when C == 0 or N_v == 0):
 *     u32 B (coefficients per block), u32 nb = ceil(N_v / B),
 *     u32 block_words[nb * C] (block-major: b * C + c),
 *     payload words in the same order, pad to 8.
 *   Coefficients of channel c in Morton (in-place) order are cut into
 *   blocks of B; each block is one RLGR stream.                           */
/* ------------------------------------------------------------------------ */
#define ORC_MAGIC 0x314E5347u

#define ORC_KLT_N 15                                 /* AC functions of degree-3 SH */
#define ORC_KLT_BYTES (3 * ORC_KLT_N * ORC_KLT_N * 4) /* three f32 15 x 15 matrices */

static int64_t header_size(int J, int C, int G, int color)
{
    int64_t h = 96 + 4 * (int64_t)(J + 1) + C;
    h = (h + 7) & ~(int64_t)7;
    h += 8 * (int64_t)G;
    if (color) h += (ORC_KLT_BYTES + 7) & ~7;
    return h;
}

/* ------------------------------------------------------------------------ */
/* Colour decorrelation of SH coefficients (Sec. 4): every SH function's RGB
 * triple goes to YUV; then one KLT per YUV channel over the 15 AC functions,
 * applied before RAHT.  Channel layout of a 56-channel 3DGS row: scale 0-2,
 * rotation 3-6, opacity 7, SH DC (R, G, B) 8-10, SH AC 11-55 as R[15] G[15]
 * B[15].  YUV is the BT.601 analogue matrix; its inverse is computed from it.
 * KLT of channel ch: K_ch (15 x 15, rows = eigenvectors of the covariance of
 * that channel's AC vector over a sample of the frame's points, by decreasing
 * eigenvalue, largest component of each made positive); a' = K_ch a.        */
/* ------------------------------------------------------------------------ */
static const double ORC_YUV[3][3] = {{0.299, 0.587, 0.114}, {-0.14713, -0.28886, 0.436}, {0.615, -0.51499, -0.10001}};

static void yuv_inverse_matrix(double inv[3][3])
{
    const double(*m)[3] = ORC_YUV;
    const double det = m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) -
                       m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
                       m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
    inv[0][0] = (m[1][1] * m[2][2] - m[1][2] * m[2][1]) / det;
    inv[0][1] = (m[0][2] * m[2][1] - m[0][1] * m[2][2]) / det;
    inv[0][2] = (m[0][1] * m[1][2] - m[0][2] * m[1][1]) / det;
    inv[1][0] = (m[1][2] * m[2][0] - m[1][0] * m[2][2]) / det;
    inv[1][1] = (m[0][0] * m[2][2] - m[0][2] * m[2][0]) / det;
    inv[1][2] = (m[0][2] * m[1][0] - m[0][0] * m[1][2]) / det;
    inv[2][0] = (m[1][0] * m[2][1] - m[1][1] * m[2][0]) / det;
    inv[2][1] = (m[0][1] * m[2][0] - m[0][0] * m[2][1]) / det;
    inv[2][2] = (m[0][0] * m[1][1] - m[0][1] * m[1][0]) / det;
}

/* channel of colour col (0 R/Y, 1 G/U, 2 B/V) of SH function k (0 = DC) */
static int sh_channel(int k, int col) { return k == 0 ? 8 + col : 11 + ORC_KLT_N * col + (k - 1); }

void orc_yuv_rows(double *A, int64_t nv, int inverse)
{
    double inv[3][3];
    yuv_inverse_matrix(inv);
    const double(*m)[3] = inverse ? (const double(*)[3])inv : ORC_YUV;
    for (int64_t i = 0; i < nv; ++i)
        for (int k = 0; k <= ORC_KLT_N; ++k) {
            double x[3], y[3];
            for (int col = 0; col < 3; ++col) x[col] = A[(size_t)i * 56 + sh_channel(k, col)];
            for (int r = 0; r < 3; ++r) y[r] = m[r][0] * x[0] + m[r][1] * x[1] + m[r][2] * x[2];
            for (int col = 0; col < 3; ++col) A[(size_t)i * 56 + sh_channel(k, col)] = y[col];
        }
}

/* a' = K a (inverse: a = K^T a') for the AC vector of each YUV channel */
void orc_klt_rows(double *A, int64_t nv, const float *K, int inverse)
{
    for (int64_t i = 0; i < nv; ++i)
        for (int ch = 0; ch < 3; ++ch) {
            double a[ORC_KLT_N], b[ORC_KLT_N];
            for (int k = 0; k < ORC_KLT_N; ++k) a[k] = A[(size_t)i * 56 + sh_channel(k + 1, ch)];
            const float *M = K + ch * ORC_KLT_N * ORC_KLT_N;
            for (int r = 0; r < ORC_KLT_N; ++r) {
                double t = 0.0;
                for (int k = 0; k < ORC_KLT_N; ++k)
                    t += (inverse ? (double)M[k * ORC_KLT_N + r] : (double)M[r * ORC_KLT_N + k]) * a[k];
                b[r] = t;
            }
            for (int k = 0; k < ORC_KLT_N; ++k) A[(size_t)i * 56 + sh_channel(k + 1, ch)] = b[k];
        }
}

/* Eigenvectors of a symmetric n x n matrix by cyclic Jacobi rotations (FP64):
 * V columns = eigenvectors, d = eigenvalues. */
static void jacobi_eig(double *S, int n, double *V, double *d)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) V[i * n + j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += S[p * n + q] * S[p * n + q];
        if (off < 1e-30) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = S[p * n + q];
                if (fabs(apq) < 1e-300) continue;
                const double theta = (S[q * n + q] - S[p * n + p]) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {  /* rows/columns p, q of S */
                    const double skp = S[k * n + p], skq = S[k * n + q];
                    S[k * n + p] = c * skp - s * skq;
                    S[k * n + q] = s * skp + c * skq;
                }
                for (int k = 0; k < n; ++k) {
                    const double spk = S[p * n + k], sqk = S[q * n + k];
                    S[p * n + k] = c * spk - s * sqk;
                    S[q * n + k] = s * spk + c * sqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - s * vkq;
                    V[k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    for (int i = 0; i < n; ++i) d[i] = S[i * n + i];
}

/* KLT matrices (f32, 3 x 15 x 15) from the first min(n, 4096) input rows. */
#define ORC_KLT_SAMPLE 4096
void orc_klt_matrices(const float *attr, int64_t n, float *K)
{
    const int N = ORC_KLT_N;
    const int64_t m = n < ORC_KLT_SAMPLE ? n : ORC_KLT_SAMPLE;
    double *rows = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1) * 56);
    for (int64_t i = 0; i < m * 56; ++i) rows[i] = (double)attr[i];
    orc_yuv_rows(rows, m, 0);
    for (int ch = 0; ch < 3; ++ch) {
        double mu[ORC_KLT_N] = {0}, S[ORC_KLT_N * ORC_KLT_N] = {0}, V[ORC_KLT_N * ORC_KLT_N], d[ORC_KLT_N];
        for (int64_t i = 0; i < m; ++i)
            for (int k = 0; k < N; ++k) mu[k] += rows[(size_t)i * 56 + sh_channel(k + 1, ch)];
        for (int k = 0; k < N; ++k) mu[k] /= (double)(m > 0 ? m : 1);
        for (int64_t i = 0; i < m; ++i)
            for (int a = 0; a < N; ++a)
                for (int b = 0; b < N; ++b)
                    S[a * N + b] += (rows[(size_t)i * 56 + sh_channel(a + 1, ch)] - mu[a]) *
                                    (rows[(size_t)i * 56 + sh_channel(b + 1, ch)] - mu[b]);
        for (int a = 0; a < N * N; ++a) S[a] /= (double)(m > 0 ? m : 1);
        jacobi_eig(S, N, V, d);
        int order[ORC_KLT_N];
        for (int k = 0; k < N; ++k) order[k] = k;
        for (int a = 0; a < N; ++a)  /* decreasing eigenvalue, stable */
            for (int b = a + 1; b < N; ++b)
                if (d[order[b]] > d[order[a]]) {
                    int t = order[a];
                    order[a] = order[b];
                    order[b] = t;
                }
        for (int r = 0; r < N; ++r) {
            const int e = order[r];
            int big = 0;
            for (int k = 1; k < N; ++k)
                if (fabs(V[k * N + e]) > fabs(V[big * N + e])) big = k;
            const double sg = V[big * N + e] < 0 ? -1.0 : 1.0;
            for (int k = 0; k < N; ++k) K[(ch * N + r) * N + k] = (float)(sg * V[k * N + e]);
        }
    }
    free(rows);
}

int64_t orc_encode_frame(const float *pos, const float *attr, int64_t n, int C, int J, int G,
                         const uint8_t *group, const double *steps, double tau, uint32_t B,
                         uint32_t chunk_syms, uint8_t *out, int64_t cap, int64_t *out_nv,
                         uint64_t *out_codes, double *out_coeff, int32_t *out_q, int color,
                         const float *klt_in, float *klt_out)
{
    if (J < 1 || J > 21 || C < 0 || (C > 0 && (G < 1 || G > 255)) || n < 0) return ORC_ERR_ARG;
    if (color && C != 56) return ORC_ERR_ARG;
    float K[ORC_KLT_BYTES / 4];
    if (C > 0 && (B == 0 || (B & (B - 1)) != 0)) return ORC_ERR_ARG;
    for (int c = 0; c < C; ++c)
        if (group[c] >= G) return ORC_ERR_ARG;
    for (int g = 0; g < G && C > 0; ++g)
        if (!(steps[g] > 0.0)) return ORC_ERR_ARG;
    double lo[3], ext;
    orc_bbox(pos, n, lo, &ext);
    uint32_t *vox = (uint32_t *)malloc(sizeof(uint32_t) * 3 * (size_t)(n > 0 ? n : 1));
    uint64_t *codes = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
    uint64_t *ucodes = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
    double *A = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * (size_t)(C > 0 ? C : 1));
    if (!vox || !codes || !ucodes || !A) {
        free(vox); free(codes); free(ucodes); free(A);
        return ORC_ERR_NOMEM;
    }
    orc_voxel_coords(pos, n, J, lo, ext, vox);
    for (int64_t i = 0; i < n; ++i) codes[i] = orc_morton(vox[3 * i], vox[3 * i + 1], vox[3 * i + 2], J);
    int64_t nv = orc_merge(codes, attr, n, C, ucodes, A, NULL);
    if (nv < 0) {
        free(vox); free(codes); free(ucodes); free(A);
        return nv;
    }
    /* distinct voxel coordinates for the level-order traversal */
    uint32_t *uvox = (uint32_t *)malloc(sizeof(uint32_t) * 3 * (size_t)(nv > 0 ? nv : 1));
    uint8_t *occ = (uint8_t *)malloc((size_t)(nv > 0 ? nv : 1) * (size_t)(J + 1));
    uint32_t *lsz = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(J + 1));
    for (int64_t i = 0; i < nv; ++i)
        orc_morton_decode(ucodes[i], J, &uvox[3 * i], &uvox[3 * i + 1], &uvox[3 * i + 2]);
    int64_t nocc = orc_octree_encode(uvox, nv, J, occ, lsz);
    int64_t occ_cap = 64 + 2 * nocc + 1024 + (nocc / 32 + 1) * 256;
    uint8_t *occsec = (uint8_t *)malloc((size_t)occ_cap);
    int64_t occ_bytes = orc_occ_section_encode(occ, nocc, chunk_syms, occsec, occ_cap);
    free(uvox);
    free(occ);
    if (occ_bytes < 0) {
        free(vox); free(codes); free(ucodes); free(A); free(lsz); free(occsec);
        return occ_bytes;
    }
    /* attributes */
    int64_t attr_bytes = 0;
    uint8_t *attrsec = NULL;
    if (color) {  /* Sec. 4: YUV on every SH function, then the per-channel KLT of the AC part */
        if (klt_in)
            memcpy(K, klt_in, sizeof(K));
        else
            orc_klt_matrices(attr, n, K);
        if (klt_out) memcpy(klt_out, K, sizeof(K));
        orc_yuv_rows(A, nv, 0);
        orc_klt_rows(A, nv, K, 0);
    }
    if (C > 0 && nv > 0) {
        double *Y = (double *)malloc(sizeof(double) * (size_t)nv * (size_t)C);
        int32_t *Q = (int32_t *)malloc(sizeof(int32_t) * (size_t)nv * (size_t)C);
        orc_raht_forward(ucodes, nv, J, C, A, Y);
        orc_quantize(Y, nv, C, group, steps, tau, Q);
        if (out_coeff) memcpy(out_coeff, Y, sizeof(double) * (size_t)nv * (size_t)C);
        if (out_q) memcpy(out_q, Q, sizeof(int32_t) * (size_t)nv * (size_t)C);
        int64_t nb = (nv + B - 1) / B;
        int64_t blk_cap = ((int64_t)B * 78 + 31) / 32 + 2;
        uint32_t *blk = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)blk_cap);
        int64_t total_cap = 8 + 4 * (int64_t)C * nb + 4 * blk_cap + 8;
        attrsec = (uint8_t *)calloc((size_t)total_cap, 1);
        put32(attrsec, B);
        put32(attrsec + 4, (uint32_t)nb);
        int64_t pw = 8 + 4 * (int64_t)C * nb;
        for (int64_t b = 0; b < nb; ++b)
            for (int c = 0; c < C; ++c) {
                int64_t s0 = b * B;
                int64_t len = (nv - s0 < (int64_t)B) ? nv - s0 : (int64_t)B;
                int64_t w = orc_rlgr_encode(Q + (size_t)s0 * C + c, len, C, blk, blk_cap);
                put32(attrsec + 8 + 4 * (b * C + c), (uint32_t)w);
                if (pw + 4 * w + 8 > total_cap) {
                    int64_t ncap = 2 * total_cap + 4 * w + 16;
                    uint8_t *grown = (uint8_t *)realloc(attrsec, (size_t)ncap);
                    memset(grown + total_cap, 0, (size_t)(ncap - total_cap));
                    attrsec = grown;
                    total_cap = ncap;
                }
                for (int64_t t = 0; t < w; ++t) put32(attrsec + pw + 4 * t, blk[t]);
                pw += 4 * w;
            }
        attr_bytes = (pw + 7) & ~(int64_t)7;
        free(blk);
        free(Y);
        free(Q);
    }
    int64_t hb = header_size(J, C, C > 0 ? G : 0, color);
    int64_t total = hb + occ_bytes + attr_bytes;
    if (out_nv) *out_nv = nv;
    if (out_codes) memcpy(out_codes, ucodes, sizeof(uint64_t) * (size_t)nv);
    if (total > cap) {
        free(vox); free(codes); free(ucodes); free(A); free(lsz); free(occsec); free(attrsec);
        return ORC_ERR_CAPACITY;
    }
    memset(out, 0, (size_t)hb);
    put32(out + 0, ORC_MAGIC);
    put32(out + 4, 1);
    put32(out + 8, (uint32_t)hb);
    put32(out + 12, (uint32_t)J);
    put32(out + 16, (uint32_t)C);
    put32(out + 20, (uint32_t)(C > 0 ? G : 0));
    put64(out + 24, (uint64_t)nv);
    for (int a = 0; a < 3; ++a) putf64(out + 32 + 8 * a, lo[a]);
    putf64(out + 56, ext);
    putf64(out + 64, tau);
    put64(out + 72, (uint64_t)occ_bytes);
    put64(out + 80, (uint64_t)attr_bytes);
    for (int d = 0; d <= J; ++d) put32(out + 96 + 4 * d, lsz[d]);
    for (int c = 0; c < C; ++c) out[96 + 4 * (J + 1) + c] = group[c];
    int64_t so = (96 + 4 * (int64_t)(J + 1) + C + 7) & ~(int64_t)7;
    for (int g = 0; g < (C > 0 ? G : 0); ++g) putf64(out + so + 8 * g, steps[g]);
    if (color) {
        put32(out + 88, 1u);  /* flags bit 0: colour decorrelation, KLT matrices follow the steps */
        memcpy(out + so + 8 * G, K, ORC_KLT_BYTES);
    }
    memcpy(out + hb, occsec, (size_t)occ_bytes);
    if (attr_bytes) memcpy(out + hb + occ_bytes, attrsec, (size_t)attr_bytes);
    free(vox); free(codes); free(ucodes); free(A); free(lsz); free(occsec); free(attrsec);
    return total;
}

/* Reads the fixed header; returns 0 or a negative error. */
int orc_peek_frame(const uint8_t *in, int64_t nbytes, int64_t *nv, int *C, int *J)
{
    if (nbytes < 96 || get32(in) != ORC_MAGIC || get32(in + 4) != 1) return ORC_ERR_CORRUPT;
    *J = (int)get32(in + 12);
    *C = (int)get32(in + 16);
    *nv = (int64_t)get64(in + 24);
    if (*J < 1 || *J > 21) return ORC_ERR_CORRUPT;
    return ORC_OK;
}

/* Decodes a frame: positions (voxel centres, float), attributes in FP64
 * (dequantised, inverse RAHT), sorted leaf codes and quantised indices.
 * Returns N_v or a negative error.  Any output pointer may be NULL.        */
int64_t orc_decode_frame(const uint8_t *in, int64_t nbytes, int64_t cap_nv, float *pos,
                         double *attr, uint64_t *codes_out, int32_t *q_out)
{
    int64_t nv;
    int C, J;
    int r = orc_peek_frame(in, nbytes, &nv, &C, &J);
    if (r) return r;
    int G = (int)get32(in + 20);
    int64_t hb = get32(in + 8);
    const uint32_t flags = get32(in + 88);
    const int color = (int)(flags & 1u);
    if ((flags & ~1u) || (color && C != 56)) return ORC_ERR_CORRUPT;
    if (hb != header_size(J, C, G, color) || hb > nbytes) return ORC_ERR_CORRUPT;
    if (nv > cap_nv) return ORC_ERR_CAPACITY;
    double lo[3];
    for (int a = 0; a < 3; ++a) lo[a] = getf64(in + 32 + 8 * a);
    double ext = getf64(in + 56), tau = getf64(in + 64);
    int64_t occ_bytes = (int64_t)get64(in + 72), attr_bytes = (int64_t)get64(in + 80);
    if (occ_bytes < 0 || attr_bytes < 0 || hb + occ_bytes + attr_bytes > nbytes) return ORC_ERR_CORRUPT;
    uint32_t lsz[22];
    int64_t nocc = 0;
    for (int d = 0; d <= J; ++d) {
        lsz[d] = get32(in + 96 + 4 * d);
        if (d < J) nocc += lsz[d];
    }
    if ((int64_t)lsz[J] != nv) return ORC_ERR_CORRUPT;
    const uint8_t *grp = in + 96 + 4 * (J + 1);
    int64_t so = (96 + 4 * (int64_t)(J + 1) + C + 7) & ~(int64_t)7;
    double steps[256];
    for (int g = 0; g < G; ++g) steps[g] = getf64(in + so + 8 * g);
    for (int c = 0; c < C; ++c)
        if (grp[c] >= G) return ORC_ERR_CORRUPT;
    uint8_t *occ = (uint8_t *)malloc((size_t)(nocc > 0 ? nocc : 1));
    int64_t got = orc_occ_section_decode(in + hb, occ_bytes, occ, nocc);
    if (got != nocc) {
        free(occ);
        return got < 0 ? got : ORC_ERR_CORRUPT;
    }
    uint64_t *codes = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(nv > 0 ? nv : 1));
    int64_t dn = orc_octree_decode(occ, nocc, J, lsz, codes, nv);
    free(occ);
    if (dn != nv) {
        free(codes);
        return dn < 0 ? dn : ORC_ERR_CORRUPT;
    }
    if (pos) orc_voxel_centres(codes, nv, J, lo, ext, pos);
    if (codes_out) memcpy(codes_out, codes, sizeof(uint64_t) * (size_t)nv);
    if (C > 0 && nv > 0) {
        const uint8_t *as = in + hb + occ_bytes;
        if (attr_bytes < 8) {
            free(codes);
            return ORC_ERR_CORRUPT;
        }
        uint32_t B = get32(as);
        int64_t nb = get32(as + 4);
        if (B == 0 || (B & (B - 1)) || nb != (nv + B - 1) / B || 8 + 4 * (int64_t)C * nb > attr_bytes) {
            free(codes);
            return ORC_ERR_CORRUPT;
        }
        int32_t *Q = (int32_t *)malloc(sizeof(int32_t) * (size_t)nv * (size_t)C);
        uint32_t *w = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(attr_bytes / 4 + 1));
        for (int64_t t = 0; t < attr_bytes / 4; ++t) w[t] = get32(as + 4 * t);
        int64_t pw = 2 + (int64_t)C * nb;
        for (int64_t b = 0; b < nb; ++b)
            for (int c = 0; c < C; ++c) {
                int64_t len = (nv - b * B < (int64_t)B) ? nv - b * B : (int64_t)B;
                int64_t bw = w[2 + b * C + c];
                if (pw + bw > attr_bytes / 4 ||
                    orc_rlgr_decode(w + pw, bw, len, C, Q + (size_t)b * B * C + c) != ORC_OK) {
                    free(Q); free(w); free(codes);
                    return ORC_ERR_CORRUPT;
                }
                pw += bw;
            }
        free(w);
        if (q_out) memcpy(q_out, Q, sizeof(int32_t) * (size_t)nv * (size_t)C);
        if (attr) {
            double *Y = (double *)malloc(sizeof(double) * (size_t)nv * (size_t)C);
            for (int64_t i = 0; i < nv; ++i)
                for (int c = 0; c < C; ++c)
                    Y[(size_t)i * C + c] = (double)Q[(size_t)i * C + c] * steps[grp[c]];
            orc_raht_inverse(codes, nv, J, C, Y, attr);
            free(Y);
            if (color) {
                float K[ORC_KLT_BYTES / 4];
                memcpy(K, in + so + 8 * G, ORC_KLT_BYTES);
                orc_klt_rows(attr, nv, K, 1);
                orc_yuv_rows(attr, nv, 1);
            }
        }
        free(Q);
    }
    (void)tau;
    free(codes);
    return nv;
}

/* ------------------------------------------------------------------------ */
/* Splat rasteriser for rendered-view quality (the paper measures rendered
 * PSNR of decoded frames; the renderer is the standard 3DGS forward pass,
 * written here from its definition).  Gaussian i of a 56-channel row: mean
 * pos[i], scale exp(attr 0-2), rotation quaternion (w, x, y, z) = attr 3-6
 * normalised, opacity sigmoid(attr 7), colour from degree-3 real SH (DC at
 * 8-10, AC function k at 11+k-1, 26+k-1, 41+k-1 for R, G, B) at the viewing
 * direction, plus 0.5, clamped at 0.
 * Camera: x_cam = R x + t (view[12] = R row-major | t), pixel (x, y) has
 * centre (x + 0.5, y + 0.5), u = fx x/z + cx, v = fy y/z + cy.  2-D covariance
 * J R S R^T J^T + 0.3 I (EWA, with the usual dilation); footprint radius
 * ceil(3 sqrt(largest eigenvalue)); tiles of 16 x 16 pixels overlapped by the
 * square [u - r, u + r] x [v - r, v + r] list the splat.  A pixel composites
 * the splats of its tile front to back (view depth, then index): alpha =
 * min(0.99, opacity exp(-d^T conic d / 2)), skipped below 1/255; stop before
 * the transmittance falls under 1e-4; background added with the remaining
 * transmittance.  Splats with z <= near or a singular 2-D covariance are
 * dropped.                                                                  */
/* ------------------------------------------------------------------------ */
#define ORC_TILE 16

typedef struct {
    double u, v, conic[3], opacity, color[3], depth;
    int tx0, tx1, ty0, ty1; /* inclusive tile range; tx0 > tx1 when empty */
    /* for the threshold check (orc_render_check): condition number of the
     * 2-D covariance, the tile ranges when the radius and centre move by a
     * hair inward (in) or outward (out), and whether z is within a hair of
     * the near plane */
    double kappa;
    int in_tx0, in_tx1, in_ty0, in_ty1, out_tx0, out_tx1, out_ty0, out_ty1;
    int near_edge;
} orc_splat;

static void sh_basis(const double d[3], double Y[16])
{
    const double x = d[0], y = d[1], z = d[2];
    const double pi = 3.14159265358979323846;
    const double c0 = 0.5 / sqrt(pi), c1 = sqrt(3.0 / (4.0 * pi));
    const double c2a = 0.5 * sqrt(15.0 / pi), c2b = 0.25 * sqrt(5.0 / pi), c2c = 0.25 * sqrt(15.0 / pi);
    const double c3a = 0.25 * sqrt(35.0 / (2.0 * pi)), c3b = 0.5 * sqrt(105.0 / pi), c3c = 0.25 * sqrt(21.0 / (2.0 * pi));
    const double c3d = 0.25 * sqrt(7.0 / pi), c3e = 0.25 * sqrt(105.0 / pi);
    Y[0] = c0;
    Y[1] = -c1 * y;
    Y[2] = c1 * z;
    Y[3] = -c1 * x;
    Y[4] = c2a * x * y;
    Y[5] = -c2a * y * z;
    Y[6] = c2b * (2.0 * z * z - x * x - y * y);
    Y[7] = -c2a * x * z;
    Y[8] = c2c * (x * x - y * y);
    Y[9] = -c3a * y * (3.0 * x * x - y * y);
    Y[10] = c3b * x * y * z;
    Y[11] = -c3c * y * (4.0 * z * z - x * x - y * y);
    Y[12] = c3d * z * (2.0 * z * z - 3.0 * x * x - 3.0 * y * y);
    Y[13] = -c3c * x * (4.0 * z * z - x * x - y * y);
    Y[14] = c3e * z * (x * x - y * y);
    Y[15] = -c3a * x * (x * x - 3.0 * y * y);
}

static int splat_prepare(const float *p, const float *a, const double view[12], double fx, double fy, double cx,
                         double cy, int W, int H, double znear, orc_splat *s)
{
    const double *R = view;
    double pc[3];
    for (int r = 0; r < 3; ++r) pc[r] = R[4 * r] * p[0] + R[4 * r + 1] * p[1] + R[4 * r + 2] * p[2] + R[4 * r + 3];
    const double z = pc[2];
    s->near_edge = fabs(z - znear) <= 1e-9 * fabs(znear);
    if (!(z > znear)) return 0;
    double q[4] = {a[3], a[4], a[5], a[6]};
    double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    if (!(qn > 0)) {
        q[0] = 1.0;
        q[1] = q[2] = q[3] = 0.0;
        qn = 1.0;
    }
    const double w = q[0] / qn, x = q[1] / qn, y = q[2] / qn, zq = q[3] / qn;
    const double Rq[9] = {1 - 2 * (y * y + zq * zq), 2 * (x * y - w * zq), 2 * (x * zq + w * y),
                          2 * (x * y + w * zq), 1 - 2 * (x * x + zq * zq), 2 * (y * zq - w * x),
                          2 * (x * zq - w * y), 2 * (y * zq + w * x), 1 - 2 * (x * x + y * y)};
    const double sc[3] = {exp(a[0]), exp(a[1]), exp(a[2])};
    double M[9], S[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) M[3 * r + c] = Rq[3 * r + c] * sc[c];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) S[3 * r + c] = M[3 * r] * M[3 * c] + M[3 * r + 1] * M[3 * c + 1] + M[3 * r + 2] * M[3 * c + 2];
    /* T = J R (2 x 3) with J the perspective Jacobian at pc */
    const double J[6] = {fx / z, 0.0, -fx * pc[0] / (z * z), 0.0, fy / z, -fy * pc[1] / (z * z)};
    double T[6];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c) T[3 * r + c] = J[3 * r] * R[c] + J[3 * r + 1] * R[4 + c] + J[3 * r + 2] * R[8 + c];
    double TS[6];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c) TS[3 * r + c] = T[3 * r] * S[c] + T[3 * r + 1] * S[3 + c] + T[3 * r + 2] * S[6 + c];
    double ca = TS[0] * T[0] + TS[1] * T[1] + TS[2] * T[2] + 0.3;
    double cb = TS[0] * T[3] + TS[1] * T[4] + TS[2] * T[5];
    double cc = TS[3] * T[3] + TS[4] * T[4] + TS[5] * T[5] + 0.3;
    const double det = ca * cc - cb * cb;
    if (!(det > 0)) return 0;
    s->conic[0] = cc / det;
    s->conic[1] = -cb / det;
    s->conic[2] = ca / det;
    const double mid = 0.5 * (ca + cc);
    const double disc = mid * mid - det;
    const double lmax = mid + sqrt(disc > 0.1 ? disc : 0.1);
    const double rad = ceil(3.0 * sqrt(lmax));
    {
        const double sd = sqrt(disc > 0 ? disc : 0.0);
        s->kappa = (mid + sd) / (mid - sd > 0 ? mid - sd : 1e-300);
    }
    s->u = fx * pc[0] / z + cx;
    s->v = fy * pc[1] / z + cy;
    s->depth = z;
    s->opacity = 1.0 / (1.0 + exp(-(double)a[7]));
    const int TX = (W + ORC_TILE - 1) / ORC_TILE, TY = (H + ORC_TILE - 1) / ORC_TILE;
    int tx0 = (int)floor((s->u - rad) / ORC_TILE), tx1 = (int)floor((s->u + rad) / ORC_TILE);
    int ty0 = (int)floor((s->v - rad) / ORC_TILE), ty1 = (int)floor((s->v + rad) / ORC_TILE);
    s->tx0 = tx0 < 0 ? 0 : tx0;
    s->tx1 = tx1 > TX - 1 ? TX - 1 : tx1;
    s->ty0 = ty0 < 0 ? 0 : ty0;
    s->ty1 = ty1 > TY - 1 ? TY - 1 : ty1;
    {  /* the same rectangle with the radius and centre moved by a hair */
        const double hr = 1e-9 * sqrt(lmax), hu = 1e-7;
        const double r_in = ceil(3.0 * (sqrt(lmax) - hr)), r_out = ceil(3.0 * (sqrt(lmax) + hr));
        int a0 = (int)floor((s->u + hu - r_in) / ORC_TILE), a1 = (int)floor((s->u - hu + r_in) / ORC_TILE);
        int b0 = (int)floor((s->v + hu - r_in) / ORC_TILE), b1 = (int)floor((s->v - hu + r_in) / ORC_TILE);
        s->in_tx0 = a0 < 0 ? 0 : a0;
        s->in_tx1 = a1 > TX - 1 ? TX - 1 : a1;
        s->in_ty0 = b0 < 0 ? 0 : b0;
        s->in_ty1 = b1 > TY - 1 ? TY - 1 : b1;
        a0 = (int)floor((s->u - hu - r_out) / ORC_TILE);
        a1 = (int)floor((s->u + hu + r_out) / ORC_TILE);
        b0 = (int)floor((s->v - hu - r_out) / ORC_TILE);
        b1 = (int)floor((s->v + hu + r_out) / ORC_TILE);
        s->out_tx0 = a0 < 0 ? 0 : a0;
        s->out_tx1 = a1 > TX - 1 ? TX - 1 : a1;
        s->out_ty0 = b0 < 0 ? 0 : b0;
        s->out_ty1 = b1 > TY - 1 ? TY - 1 : b1;
    }
    /* colour: degree-3 SH at the direction from the camera centre (-R^T t) */
    double cam[3], d[3];
    for (int c = 0; c < 3; ++c) cam[c] = -(R[c] * R[3] + R[4 + c] * R[7] + R[8 + c] * R[11]);
    for (int c = 0; c < 3; ++c) d[c] = (double)p[c] - cam[c];
    const double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int c = 0; c < 3; ++c) d[c] /= (dn > 0 ? dn : 1.0);
    double Y[16];
    sh_basis(d, Y);
    for (int col = 0; col < 3; ++col) {
        double v = Y[0] * a[8 + col];
        for (int k = 1; k < 16; ++k) v += Y[k] * a[11 + 15 * col + (k - 1)];
        v += 0.5;
        s->color[col] = v > 0 ? v : 0;
    }
    return 1;
}

typedef struct {
    double depth;
    int64_t idx;
} orc_depth_key;

static int depth_cmp(const void *x, const void *y)
{
    const orc_depth_key *a = (const orc_depth_key *)x, *b = (const orc_depth_key *)y;
    if (a->depth < b->depth) return -1;
    if (a->depth > b->depth) return 1;
    return (a->idx > b->idx) - (a->idx < b->idx);
}

static int covers(int tx, int ty, int x0, int x1, int y0, int y1) { return tx >= x0 && tx <= x1 && ty >= y0 && ty <= y1; }

/* Renders n Gaussians into image[H][W][3] (FP64).  When flag and tol are
 * given, it also marks (flag = 1) every pixel whose value hangs on a decision
 * taken within a hair of its threshold, where a renderer computing in FP32
 * may legitimately decide the other way:
 *   - some splat's alpha within relative 1e-5 of the 1/255 cut;
 *   - the transmittance after a splat within relative 1e-4 of the 1e-4 stop;
 *   - a splat whose tile rectangle covers the pixel's tile only for a radius
 *     or centre moved by a hair (and that reaches alpha 1/255 there);
 *   - two splats passing the alpha cut whose distinct depths round to the
 *     same FP32 value (their order is then the index order in FP32);
 *   - a splat exactly at the pixel centre with a rounded-up positive
 *     exponent, or a splat at the near plane;
 * and gives every other pixel a first-order bound tol on the error of an
 * FP32 evaluation of the same pixel from FP32-rounded per-splat values
 * (u, v to FP32 of their offsets, conic, opacity, colour):
 *   tol = sum_k T_k (|c_k| + c_max) alpha_k e_k + 2^-24 (6 + 6 n) c_max,
 * where the sum runs over the n composited splats, T_k is the transmittance
 * in front of splat k, c_max the largest colour value among them and the
 * background, and e_k = 2^-24 (8 + 8 p_k (1 + sqrt(kappa_k))) bounds the
 * relative error of alpha_k (exponential and opacity rounding, and the
 * exponent p_k = |d^T conic d| / 2 evaluated as a sum of squares of a
 * Cholesky factor whose conditioning is that of the 2-D covariance,
 * kappa_k).  d C / d alpha_k is bounded by T_k (|c_k| + c_max): the splat's
 * own colour and, through (1 - alpha_k), everything behind it.             */
static int render_impl(const float *pos, const float *attr, int64_t n, const double view[12], double fx, double fy,
                       double cx, double cy, int W, int H, double znear, const double bg[3], double *image,
                       uint8_t *flag, double *tol)
{
    orc_splat *sp = (orc_splat *)malloc(sizeof(orc_splat) * (size_t)(n > 0 ? n : 1));
    orc_depth_key *ord = (orc_depth_key *)malloc(sizeof(orc_depth_key) * (size_t)(n > 0 ? n : 1));
    if (!sp || !ord) {
        free(sp);
        free(ord);
        return ORC_ERR_NOMEM;
    }
    const int check = flag != NULL && tol != NULL;
    const double u24 = ldexp(1.0, -24);
    int64_t m = 0, near_edge = 0;
    for (int64_t i = 0; i < n; ++i) {
        const int ok = splat_prepare(pos + 3 * i, attr + 56 * i, view, fx, fy, cx, cy, W, H, znear, &sp[i]);
        near_edge |= sp[i].near_edge;
        if (ok && (check ? sp[i].out_tx0 <= sp[i].out_tx1 && sp[i].out_ty0 <= sp[i].out_ty1
                         : sp[i].tx0 <= sp[i].tx1 && sp[i].ty0 <= sp[i].ty1)) {
            ord[m].depth = sp[i].depth;
            ord[m].idx = i;
            ++m;
        }
    }
    qsort(ord, (size_t)m, sizeof(orc_depth_key), depth_cmp);
    for (int py = 0; py < H; ++py)
        for (int px = 0; px < W; ++px) {
            const int tx = px / ORC_TILE, ty = py / ORC_TILE;
            double T = 1.0, col[3] = {0, 0, 0};
            const double fxp = px + 0.5, fyp = py + 0.5;
            int marked = near_edge != 0, np = 0, passed = 0;
            double cmax = fmax(fabs(bg[0]), fmax(fabs(bg[1]), fabs(bg[2])));
            double s0 = 0.0, s1 = 0.0, relT = 0.0;  /* sum T a e, sum T a e |c|, relative error bound of T */
            float prev_depth = -1.0f;
            double prev_depth64 = -1.0;
            for (int64_t k = 0; k < m; ++k) {
                const orc_splat *s = &sp[ord[k].idx];
                const int in_nominal = covers(tx, ty, s->tx0, s->tx1, s->ty0, s->ty1);
                if (!in_nominal && !(check && covers(tx, ty, s->out_tx0, s->out_tx1, s->out_ty0, s->out_ty1))) continue;
                const double dx = s->u - fxp, dy = s->v - fyp;
                const double power = -0.5 * (s->conic[0] * dx * dx + s->conic[2] * dy * dy) - s->conic[1] * dx * dy;
                double alpha = s->opacity * exp(power > 0 ? 0.0 : power);
                if (alpha > 0.99) alpha = 0.99;
                const double ek = u24 * (8.0 + 8.0 * fabs(power) * (1.0 + sqrt(s->kappa)));
                if (check) {
                    const int marginal = !covers(tx, ty, s->in_tx0, s->in_tx1, s->in_ty0, s->in_ty1);
                    if (marginal && alpha >= (1.0 / 255.0) * (1.0 - 2.0 * ek - 1e-6)) marked = 1;
                    if (fabs(alpha - 1.0 / 255.0) <= (1.0 / 255.0) * (2.0 * ek + 1e-6)) marked = 1;
                    if (power > 0 && alpha >= 1.0 / 255.0) marked = 1;
                }
                if (!in_nominal || power > 0) continue;
                if (alpha < 1.0 / 255.0) continue;
                if (check) {
                    const float fd = (float)s->depth;
                    if (passed > 0 && fd == prev_depth && s->depth != prev_depth64) marked = 1;
                    prev_depth = fd;
                    prev_depth64 = s->depth;
                    ++passed;
                }
                const double tn = T * (1.0 - alpha);
                if (check) {
                    relT += alpha * ek / (1.0 - alpha) + 2.0 * u24;
                    if (fabs(tn - 1e-4) <= 1e-4 * (2.0 * relT + 1e-6)) marked = 1;
                }
                if (tn < 1e-4) break;
                for (int c = 0; c < 3; ++c) col[c] += s->color[c] * alpha * T;
                if (check) {
                    const double ck = fmax(s->color[0], fmax(s->color[1], s->color[2]));
                    cmax = fmax(cmax, ck);
                    s0 += T * alpha * ek;
                    s1 += T * alpha * ek * ck;
                    ++np;
                }
                T = tn;
            }
            for (int c = 0; c < 3; ++c) image[((size_t)py * W + px) * 3 + c] = col[c] + T * bg[c];
            if (check) {
                flag[(size_t)py * W + px] = (uint8_t)marked;
                tol[(size_t)py * W + px] = s1 + cmax * s0 + u24 * (6.0 + 6.0 * np) * cmax;
            }
        }
    free(sp);
    free(ord);
    return ORC_OK;
}

int orc_render(const float *pos, const float *attr, int64_t n, const double view[12], double fx, double fy,
               double cx, double cy, int W, int H, double znear, const double bg[3], double *image)
{
    return render_impl(pos, attr, n, view, fx, fy, cx, cy, W, H, znear, bg, image, NULL, NULL);
}

/* orc_render plus the per-pixel threshold flags and error bounds above. */
int orc_render_check(const float *pos, const float *attr, int64_t n, const double view[12], double fx, double fy,
                     double cx, double cy, int W, int H, double znear, const double bg[3], double *image,
                     uint8_t *flag, double *tol)
{
    if (!flag || !tol) return ORC_ERR_ARG;
    return render_impl(pos, attr, n, view, fx, fy, cx, cy, W, H, znear, bg, image, flag, tol);
}

/* The 16 real SH basis values (degrees 0-3) at a unit direction (tests). */
void orc_sh_basis(const double d[3], double Y[16]) { sh_basis(d, Y); }
