/*
 * CPU oracle for exact (alpha, beta)-cores of bipartite graphs.
 *
 * TEST INFRASTRUCTURE ONLY. This is a plain, slow, single-threaded restatement of the paper's
 * definitions, used by the test-suite, the smoke check and the benchmark's CPU-baseline leg to
 * check and time the CUDA library. The library's product path never links, loads or calls it,
 * and this file shares no code with the CUDA sources.
 *
 * Vertex ids are unified as in Section 4.1 of the paper: U vertex u is u, V (lower-layer)
 * vertex v is nU + v, so the layer of x is the range test x < nU.
 *
 * Functions and what they follow:
 *   orc_build_csr     - CSR storage of both layers (Section 3), each row sorted ascending.
 *   orc_peel_csr      - Definition 1 reached by the peeling method ("Online", Section 3.1):
 *                       remove every upper vertex with degree < alpha and every lower vertex
 *                       with degree < beta, with their edges, until no vertex violates.
 *   orc_core_numbers  - Definition 2 core numbers, by the Batagelj-Zaversnik bucket algorithm.
 *   orc_replay        - the on-the-fly query problem (Section 3): apply edge updates in order,
 *                       and at the requested steps peel the updated graph from scratch and
 *                       report whether both endpoints of the update lie in the target core.
 *   orc_components    - connected components of the graph (the labels GFQ keeps, Section 5),
 *                       by breadth-first search from each unvisited vertex in increasing id
 *                       order, so each component is labelled by its smallest unified id.
 *
 * Return codes match the library's: 0 ok, -1 invalid argument, -3 out of memory,
 * -4 edge already present, -5 edge absent.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-3)
#define ORC_EEXIST (-4)
#define ORC_ENOENT (-5)

/* ---------------------------------------------------------------------------------------- */
/* CSR of both layers, rows sorted, by three counting passes (no comparison sort needed):     */
/* unsorted U rows; then V rows filled by walking U rows in u order (sorted by u); then U     */
/* rows refilled by walking V rows in v order (sorted by v).                                  */
/* ---------------------------------------------------------------------------------------- */
int orc_build_csr(int32_t nU, int32_t nV, int64_t m, const int32_t *eu, const int32_t *ev,
                  int64_t *off, int32_t *adj)
{
    if (nU < 0 || nV < 0 || m < 0) return ORC_EINVAL;
    for (int64_t i = 0; i < m; ++i)
        if (eu[i] < 0 || eu[i] >= nU || ev[i] < 0 || ev[i] >= nV) return ORC_EINVAL;

    int64_t n = (int64_t)nU + nV;
    int64_t *offU = calloc((size_t)nU + 1, sizeof(int64_t));
    int64_t *offV = calloc((size_t)nV + 1, sizeof(int64_t));
    int64_t *cur = malloc(((size_t)(nU > nV ? nU : nV) + 1) * sizeof(int64_t));
    int32_t *rowsU = malloc((size_t)(m ? m : 1) * sizeof(int32_t));
    int32_t *rowsV = malloc((size_t)(m ? m : 1) * sizeof(int32_t));
    if (!offU || !offV || !cur || !rowsU || !rowsV) {
        free(offU); free(offV); free(cur); free(rowsU); free(rowsV);
        return ORC_ENOMEM;
    }
    for (int64_t i = 0; i < m; ++i) { offU[eu[i] + 1]++; offV[ev[i] + 1]++; }
    for (int32_t u = 0; u < nU; ++u) offU[u + 1] += offU[u];
    for (int32_t v = 0; v < nV; ++v) offV[v + 1] += offV[v];

    /* pass 1: unsorted U rows */
    for (int32_t u = 0; u < nU; ++u) cur[u] = offU[u];
    for (int64_t i = 0; i < m; ++i) rowsU[cur[eu[i]]++] = ev[i];
    /* pass 2: V rows, sorted by u because u is walked in increasing order */
    for (int32_t v = 0; v < nV; ++v) cur[v] = offV[v];
    for (int32_t u = 0; u < nU; ++u)
        for (int64_t j = offU[u]; j < offU[u + 1]; ++j) rowsV[cur[rowsU[j]]++] = u;
    /* pass 3: U rows again, sorted by v */
    for (int32_t u = 0; u < nU; ++u) cur[u] = offU[u];
    for (int32_t v = 0; v < nV; ++v)
        for (int64_t j = offV[v]; j < offV[v + 1]; ++j) rowsU[cur[rowsV[j]]++] = v;

    int rc = ORC_OK;
    for (int32_t u = 0; u < nU && rc == ORC_OK; ++u)
        for (int64_t j = offU[u] + 1; j < offU[u + 1]; ++j)
            if (rowsU[j] == rowsU[j - 1]) { rc = ORC_EEXIST; break; }

    if (rc == ORC_OK) {
        for (int32_t u = 0; u <= nU; ++u) off[u] = offU[u];
        for (int32_t v = 1; v <= nV; ++v) off[nU + v] = m + offV[v];
        for (int64_t j = 0; j < m; ++j) adj[j] = nU + rowsU[j];
        for (int64_t j = 0; j < m; ++j) adj[m + j] = rowsV[j];
    }
    (void)n;
    free(offU); free(offV); free(cur); free(rowsU); free(rowsV);
    return rc;
}

/* ---------------------------------------------------------------------------------------- */
/* Peeling to the (alpha, beta)-core over rows given as (pointer, length) per unified vertex. */
/* deg[x] starts at |N(x)|; every violator (deg < alpha on U, deg < beta on V) is marked      */
/* removed and queued; popping x lowers the degree of each neighbour that is still present     */
/* and queues a neighbour the moment it violates. Survivors form the core (Definition 1).     */
/* ---------------------------------------------------------------------------------------- */
static int peel_rows(int32_t nU, int64_t n, int32_t *const *rows, const int64_t *len,
                     int32_t alpha, int32_t beta, uint8_t *alive)
{
    int64_t *deg = malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    int32_t *queue = malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    uint8_t *removed = calloc((size_t)(n ? n : 1), 1);
    if (!deg || !queue || !removed) { free(deg); free(queue); free(removed); return ORC_ENOMEM; }

    int64_t qh = 0, qt = 0;
    for (int64_t x = 0; x < n; ++x) {
        deg[x] = len[x];
        int64_t thr = x < nU ? alpha : beta;
        if (deg[x] < thr) { removed[x] = 1; queue[qt++] = (int32_t)x; }
    }
    while (qh < qt) {
        int32_t x = queue[qh++];
        for (int64_t j = 0; j < len[x]; ++j) {
            int32_t y = rows[x][j];
            if (removed[y]) continue;
            deg[y] -= 1;
            int64_t thr = y < nU ? alpha : beta;
            if (deg[y] < thr) { removed[y] = 1; queue[qt++] = y; }
        }
    }
    for (int64_t x = 0; x < n; ++x) alive[x] = removed[x] ? 0 : 1;
    free(deg); free(queue); free(removed);
    return ORC_OK;
}

int orc_peel_csr(int32_t nU, int32_t nV, const int64_t *off, const int32_t *adj,
                 int32_t alpha, int32_t beta, uint8_t *alive)
{
    if (nU < 0 || nV < 0 || alpha < 0 || beta < 0) return ORC_EINVAL;
    int64_t n = (int64_t)nU + nV;
    int32_t **rows = malloc((size_t)(n ? n : 1) * sizeof(int32_t *));
    int64_t *len = malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    if (!rows || !len) { free(rows); free(len); return ORC_ENOMEM; }
    for (int64_t x = 0; x < n; ++x) {
        rows[x] = (int32_t *)(adj + off[x]);
        len[x] = off[x + 1] - off[x];
    }
    int rc = peel_rows(nU, n, rows, len, alpha, beta, alive);
    free(rows); free(len);
    return rc;
}

/* ---------------------------------------------------------------------------------------- */
/* Core numbers (Definition 2): the largest k such that x lies in the (k,k)-core, i.e. the     */
/* ordinary k-core number of the graph read as unipartite. Batagelj-Zaversnik: vertices kept   */
/* in degree-bucket order; processing vertices in that order fixes each one's core number and  */
/* moves each higher-degree neighbour down one bucket.                                         */
/* ---------------------------------------------------------------------------------------- */
int orc_core_numbers(int32_t nU, int32_t nV, const int64_t *off, const int32_t *adj, int32_t *core)
{
    int64_t n = (int64_t)nU + nV;
    if (n == 0) return ORC_OK;
    int64_t md = 0;
    for (int64_t x = 0; x < n; ++x) {
        int64_t d = off[x + 1] - off[x];
        core[x] = (int32_t)d;
        if (d > md) md = d;
    }
    int64_t *bin = calloc((size_t)md + 1, sizeof(int64_t));
    int64_t *pos = malloc((size_t)n * sizeof(int64_t));
    int32_t *vert = malloc((size_t)n * sizeof(int32_t));
    if (!bin || !pos || !vert) { free(bin); free(pos); free(vert); return ORC_ENOMEM; }
    for (int64_t x = 0; x < n; ++x) bin[core[x]]++;
    int64_t start = 0;
    for (int64_t d = 0; d <= md; ++d) { int64_t c = bin[d]; bin[d] = start; start += c; }
    for (int64_t x = 0; x < n; ++x) { pos[x] = bin[core[x]]; vert[pos[x]] = (int32_t)x; bin[core[x]]++; }
    for (int64_t d = md; d >= 1; --d) bin[d] = bin[d - 1];
    bin[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int32_t x = vert[i];
        for (int64_t j = off[x]; j < off[x + 1]; ++j) {
            int32_t y = adj[j];
            if (core[y] > core[x]) {
                int64_t dy = core[y], py = pos[y], pw = bin[dy];
                int32_t w = vert[pw];
                if (y != w) { pos[y] = pw; vert[py] = w; pos[w] = py; vert[pw] = y; }
                bin[dy]++;
                core[y]--;
            }
        }
    }
    free(bin); free(pos); free(vert);
    return ORC_OK;
}

/* ---------------------------------------------------------------------------------------- */
/* Dynamic graph replay for the on-the-fly query problem. Adjacency is one growable array per  */
/* unified vertex. Op k inserts (op 0) or deletes (op 1) the edge (qu[k], qv[k]); inserting a  */
/* present edge gives -4 and deleting an absent one -5, both without changing the graph. When */
/* check[k] is set, the (alpha[k], beta[k])-core of the graph after op k is computed from      */
/* scratch and answer[k] = 1 iff both endpoints are in it (bits[k]: bit 0 = u in core,         */
/* bit 1 = v in core); otherwise answer[k] = -1.                                               */
/* ---------------------------------------------------------------------------------------- */
typedef struct { int32_t *a; int64_t len, cap; } orow;

static int row_push(orow *r, int32_t y)
{
    if (r->len == r->cap) {
        int64_t nc = r->cap ? 2 * r->cap : 4;
        int32_t *na = realloc(r->a, (size_t)nc * sizeof(int32_t));
        if (!na) return ORC_ENOMEM;
        r->a = na; r->cap = nc;
    }
    r->a[r->len++] = y;
    return ORC_OK;
}

static int64_t row_find(const orow *r, int32_t y)
{
    for (int64_t j = 0; j < r->len; ++j) if (r->a[j] == y) return j;
    return -1;
}

int orc_replay(int32_t nU, int32_t nV, int64_t m, const int32_t *eu, const int32_t *ev,
               int64_t nops, const int8_t *op, const int32_t *qu, const int32_t *qv,
               const int32_t *alpha, const int32_t *beta, const uint8_t *check,
               int8_t *answer, uint8_t *bits, int32_t *status)
{
    if (nU < 0 || nV < 0 || m < 0 || nops < 0) return ORC_EINVAL;
    int64_t n = (int64_t)nU + nV;
    orow *g = calloc((size_t)(n ? n : 1), sizeof(orow));
    int32_t **rows = malloc((size_t)(n ? n : 1) * sizeof(int32_t *));
    int64_t *len = malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    uint8_t *alive = malloc((size_t)(n ? n : 1));
    int rc = ORC_OK;
    if (!g || !rows || !len || !alive) { rc = ORC_ENOMEM; goto done; }
    for (int64_t i = 0; i < m && rc == ORC_OK; ++i) {
        if (eu[i] < 0 || eu[i] >= nU || ev[i] < 0 || ev[i] >= nV) { rc = ORC_EINVAL; break; }
        int32_t x = eu[i], y = nU + ev[i];
        rc = row_push(&g[x], y);
        if (rc == ORC_OK) rc = row_push(&g[y], x);
    }
    for (int64_t k = 0; k < nops && rc == ORC_OK; ++k) {
        if (qu[k] < 0 || qu[k] >= nU || qv[k] < 0 || qv[k] >= nV) { rc = ORC_EINVAL; break; }
        int32_t x = qu[k], y = nU + qv[k];
        int64_t jx = row_find(&g[x], y);
        status[k] = ORC_OK;
        if (op[k] == 0) {
            if (jx >= 0) status[k] = ORC_EEXIST;
            else {
                rc = row_push(&g[x], y);
                if (rc == ORC_OK) rc = row_push(&g[y], x);
            }
        } else {
            if (jx < 0) status[k] = ORC_ENOENT;
            else {
                int64_t jy = row_find(&g[y], x);
                g[x].a[jx] = g[x].a[--g[x].len];
                g[y].a[jy] = g[y].a[--g[y].len];
            }
        }
        answer[k] = -1;
        bits[k] = 0;
        if (rc == ORC_OK && check[k]) {
            for (int64_t z = 0; z < n; ++z) { rows[z] = g[z].a; len[z] = g[z].len; }
            rc = peel_rows(nU, n, rows, len, alpha[k], beta[k], alive);
            if (rc == ORC_OK) {
                bits[k] = (uint8_t)(alive[x] | (alive[y] << 1));
                answer[k] = (int8_t)(alive[x] && alive[y]);
            }
        }
    }
done:
    if (g) for (int64_t z = 0; z < n; ++z) free(g[z].a);
    free(g); free(rows); free(len); free(alive);
    return rc;
}

/* ---------------------------------------------------------------------------------------- */
/* Connected components: breadth-first search from every vertex not yet reached, taking start */
/* vertices in increasing unified id; every vertex reached gets the start's id as its label,  */
/* which is then the smallest id in its component. Returns the component count in *ncomp.     */
/* ---------------------------------------------------------------------------------------- */
int orc_components(int32_t nU, int32_t nV, const int64_t *off, const int32_t *adj, int32_t *label,
                   int64_t *ncomp)
{
    if (nU < 0 || nV < 0) return ORC_EINVAL;
    int64_t n = (int64_t)nU + nV;
    int32_t *queue = malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    if (!queue) return ORC_ENOMEM;
    for (int64_t x = 0; x < n; ++x) label[x] = -1;
    int64_t count = 0;
    for (int64_t s = 0; s < n; ++s) {
        if (label[s] >= 0) continue;
        count++;
        int64_t head = 0, tail = 0;
        label[s] = (int32_t)s;
        queue[tail++] = (int32_t)s;
        while (head < tail) {
            int32_t x = queue[head++];
            for (int64_t i = off[x]; i < off[x + 1]; ++i) {
                int32_t y = adj[i];
                if (label[y] < 0) {
                    label[y] = (int32_t)s;
                    queue[tail++] = y;
                }
            }
        }
    }
    free(queue);
    *ncomp = count;
    return ORC_OK;
}
