/*
 * oracle.c -- TEST INFRASTRUCTURE ONLY.  The plain, slow, CPU definition of
 * what the forest-classification path computes, used to check the GPU library
 * and as the timed CPU baseline.  Only tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header or
 * table with the GPU library.
 *
 * Functions and the passages they follow:
 *
 *  or_predict      Section III: a forest of T trees, each internal node a split
 *                  with two children, each leaf one class label.  Every
 *                  observation walks root to leaf in every tree; x[f] <= t goes
 *                  left (the paper does not state the comparison; this is the
 *                  reading used throughout), NaN goes right.  Votes are per-class
 *                  leaf counts; the class is the argmax, lowest class index on
 *                  ties (the paper is silent on ties).  Also counts visited
 *                  internal nodes (the "depth of test" of Table I).
 *
 *  or_layout_*     Section III-A and Fig. 1, the paper's own layouts, each an
 *                  array of nodes with explicit child indices:
 *                    BF    breadth-first per tree;
 *                    DF    depth-first (pre-order, left first) per tree;
 *                    DF-   DF with leaves replaced by one shared class node
 *                          per class, appended after the tree's internal nodes;
 *                    Stat  DF- where, at each parent, the child of larger
 *                          training cardinality is placed adjacent (left on
 *                          ties) and an internal child is always adjacent when
 *                          its sibling is a leaf;
 *                    Bin   B consecutive trees per bin; the internal nodes of
 *                          levels 0..d of all trees of the bin are interleaved
 *                          level by level (tree-major within a level, breadth-
 *                          first within a tree), deeper nodes follow tree by
 *                          tree in Stat order, and one class node per class
 *                          closes the bin.  Depth 0 interleaves the roots only
 *                          (Fig. 2 caption).
 *                  The Bin layout is evaluated as in Section III-B (Bin+):
 *                  all trees of a bin advance one level per round-robin sweep.
 *                  Layouts change node order only (Section III-A: the
 *                  optimisations do not modify the prediction algorithm), so
 *                  every layout must give the same leaf per (observation, tree).
 *
 *  or_eu_stat      Section III-A, expected utility of a cache load:
 *                  EU = 1 + b(1 + b(1 + b)), b = max(LC, RC) / PN.
 *  or_forest_stats Table I quantities: mean internal nodes per tree, largest
 *                  tree depth, mean bias max(LC, RC) / PN over internal nodes
 *                  (the mean depth of test is or_predict's visit count / (n T)).
 *
 * Compiled without -ffast-math (IEEE comparisons) and with -ffp-contract=off.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------ plain walk */

/* Walk one tree from its root; returns the tree-local leaf id and adds the
 * number of internal nodes evaluated to *visits. */
static int32_t walk(const int32_t *left, const int32_t *right, const int32_t *feature, const float *threshold,
                    const float *x, int64_t *visits) {
    int32_t node = 0;
    while (left[node] >= 0) {
        const float v = x[feature[node]];
        node = (v <= threshold[node]) ? left[node] : right[node];
        ++*visits;
    }
    return node;
}

/* Classify n observations.  Forest arrays are concatenated per tree with
 * node_begin[T+1] offsets; child ids are tree-local.  Any output may be NULL.
 *   out_leaf  [n][T]  tree-local leaf id
 *   out_votes [n][C]  leaf-class counts
 *   out_class [n]     argmax of votes, lowest index on ties
 *   out_visits        total internal nodes evaluated
 * Returns 0, or -1 on bad arguments. */
int or_predict(int32_t T, int32_t F, int32_t C, const int64_t *node_begin, const int32_t *left, const int32_t *right,
               const int32_t *feature, const float *threshold, const int32_t *leaf_class, const float *X, int64_t n,
               int32_t n_threads, int32_t *out_leaf, uint32_t *out_votes, int32_t *out_class, int64_t *out_visits) {
    if (T < 0 || F < 1 || C < 1 || n < 0) return -1;
    if (!out_votes && C > 1024) return -1;
    int64_t total = 0;
    if (n_threads < 1) n_threads = 1;
#pragma omp parallel for num_threads(n_threads) schedule(dynamic, 64) reduction(+ : total)
    for (int64_t i = 0; i < n; ++i) {
        const float *x = X + i * F;
        uint32_t votes_local[1024];
        uint32_t *votes = out_votes ? out_votes + i * C : votes_local;
        for (int32_t c = 0; c < C; ++c) votes[c] = 0;
        int64_t visits = 0;
        for (int32_t t = 0; t < T; ++t) {
            const int64_t b = node_begin[t];
            int32_t leaf = walk(left + b, right + b, feature + b, threshold + b, x, &visits);
            if (out_leaf) out_leaf[i * T + t] = leaf;
            votes[leaf_class[b + leaf]] += 1;
        }
        if (out_class) {
            int32_t best = 0;
            for (int32_t c = 1; c < C; ++c)
                if (votes[c] > votes[best]) best = c;
            out_class[i] = best;
        }
        total += visits;
    }
    if (out_visits) *out_visits = total;
    return 0;
}

/* --------------------------------------------------------- paper layouts */

enum { OR_BF = 0, OR_DF = 1, OR_DFM = 2, OR_STAT = 3, OR_BIN = 4 };

typedef struct {
    int32_t feature;   /* -1 marks a leaf (BF, DF) or a class node (DF-, Stat, Bin) */
    float threshold;
    int32_t child[2];  /* indices into the layout array */
    int32_t cls;       /* class of a leaf / class node */
    int32_t orig;      /* tree-local id of this node in the forest (-1 for shared class nodes) */
} or_node;

typedef struct {
    int32_t kind, T, C, bin_size, depth;
    int64_t n_nodes, cap;
    or_node *nodes;
    int32_t *root;      /* [T] index of each tree's root in nodes */
    int32_t *tree_of;   /* [n_nodes] tree index of each node (-1 for shared class nodes) */
} or_layout;

static int32_t lay_push(or_layout *L, or_node nd, int32_t tree) {
    if (L->n_nodes == L->cap) {
        int64_t nc = L->cap ? 2 * L->cap : 1024;
        or_node *p = realloc(L->nodes, sizeof(or_node) * (size_t)nc);
        int32_t *q = realloc(L->tree_of, sizeof(int32_t) * (size_t)nc);
        if (p) L->nodes = p;
        if (q) L->tree_of = q;
        if (!p || !q) return -1;
        L->cap = nc;
    }
    L->nodes[L->n_nodes] = nd;
    L->tree_of[L->n_nodes] = tree;
    return (int32_t)L->n_nodes++;
}

typedef struct {
    const int64_t *node_begin;
    const int32_t *left, *right, *feature, *leaf_class;
    const float *threshold;
    const int64_t *card;
} forest_ref;

/* Stat child order: returns 1 if the right child goes first (adjacent). */
static int stat_right_first(const forest_ref *f, int64_t b, int32_t v) {
    int32_t l = f->left[b + v], r = f->right[b + v];
    int l_int = f->left[b + l] >= 0, r_int = f->left[b + r] >= 0;
    if (l_int != r_int) return r_int; /* internal child adjacent to its parent */
    return f->card[b + r] > f->card[b + l]; /* larger cardinality adjacent; left on ties */
}

/* Place the subtree of tree-local node v of tree t in pre-order (DF) or
 * hot-first pre-order (Stat), with leaves either kept (DF) or redirected to
 * class nodes cls_node[] (DF-, Stat).  Returns the index of v's node in L. */
static int32_t place_df(or_layout *L, const forest_ref *f, int32_t t, int32_t v, int stat, const int32_t *cls_node) {
    const int64_t b = f->node_begin[t];
    if (f->left[b + v] < 0) {
        if (cls_node) return cls_node[f->leaf_class[b + v]];
        or_node nd = {-1, 0.0f, {-1, -1}, f->leaf_class[b + v], v};
        return lay_push(L, nd, t);
    }
    or_node nd = {f->feature[b + v], f->threshold[b + v], {-1, -1}, -1, v};
    int32_t me = lay_push(L, nd, t);
    if (me < 0) return -1;
    int first = stat ? stat_right_first(f, b, v) : 0;
    int32_t kids[2] = {f->left[b + v], f->right[b + v]};
    int32_t a = place_df(L, f, t, kids[first], stat, cls_node);
    int32_t c = place_df(L, f, t, kids[1 - first], stat, cls_node);
    if (a == -1 || c == -1) return -1; /* values <= -2 are class-node placeholders */
    L->nodes[me].child[first] = a;
    L->nodes[me].child[1 - first] = c;
    return me;
}

/* Class nodes for classes 0..C-1 appended at the current end of the array. */
static int append_class_nodes(or_layout *L, int32_t C, int32_t tree, int32_t *cls_node) {
    for (int32_t c = 0; c < C; ++c) {
        or_node nd = {-1, 0.0f, {-1, -1}, c, -1};
        cls_node[c] = lay_push(L, nd, tree);
        if (cls_node[c] < 0) return -1;
    }
    return 0;
}

static int build_bf_tree(or_layout *L, const forest_ref *f, int32_t t) {
    const int64_t b = f->node_begin[t];
    const int64_t m = f->node_begin[t + 1] - b;
    int32_t *queue = malloc(sizeof(int32_t) * (size_t)m);
    int32_t *pos = malloc(sizeof(int32_t) * (size_t)m);
    if (!queue || !pos) { free(queue); free(pos); return -1; }
    int64_t head = 0, tail = 0;
    queue[tail++] = 0;
    while (head < tail) {
        int32_t v = queue[head++];
        or_node nd = {f->left[b + v] >= 0 ? f->feature[b + v] : -1, f->left[b + v] >= 0 ? f->threshold[b + v] : 0.0f,
                      {-1, -1}, f->left[b + v] >= 0 ? -1 : f->leaf_class[b + v], v};
        pos[v] = lay_push(L, nd, t);
        if (pos[v] < 0) { free(queue); free(pos); return -1; }
        if (f->left[b + v] >= 0) {
            queue[tail++] = f->left[b + v];
            queue[tail++] = f->right[b + v];
        }
    }
    for (int64_t k = 0; k < tail; ++k) {
        int32_t v = queue[k];
        if (f->left[b + v] >= 0) {
            L->nodes[pos[v]].child[0] = pos[f->left[b + v]];
            L->nodes[pos[v]].child[1] = pos[f->right[b + v]];
        }
    }
    L->root[t] = pos[0];
    free(queue);
    free(pos);
    return 0;
}

/* Bin of trees [t0, t1): interleaved levels 0..d, then Stat per tree, then
 * class nodes.  Children below the interleaved block are placed per tree
 * after the block, in the order the block's nodes reference them. */
static int build_bin(or_layout *L, const forest_ref *f, int32_t t0, int32_t t1, int32_t d, int32_t C) {
    const int32_t nb = t1 - t0;
    const int64_t bin_start = L->n_nodes;
    /* level lists of internal nodes per tree, breadth-first, for levels 0..d */
    int64_t total = 0;
    for (int32_t t = t0; t < t1; ++t) total += f->node_begin[t + 1] - f->node_begin[t];
    int32_t *lvl_nodes = malloc(sizeof(int32_t) * (size_t)(total + 1));
    int32_t *lvl_tree = malloc(sizeof(int32_t) * (size_t)(total + 1));
    int32_t *where = malloc(sizeof(int32_t) * (size_t)(total + 1)); /* layout index, per bin-local node */
    int64_t *boff = malloc(sizeof(int64_t) * (size_t)(nb + 1));
    int32_t *frontier = malloc(sizeof(int32_t) * (size_t)(total + 1));
    int32_t *next = malloc(sizeof(int32_t) * (size_t)(total + 1));
    int32_t *cls_node = malloc(sizeof(int32_t) * (size_t)C);
    int rc = -1;
    if (!lvl_nodes || !lvl_tree || !where || !boff || !frontier || !next || !cls_node) goto done;
    boff[0] = 0;
    for (int32_t k = 0; k < nb; ++k) boff[k + 1] = boff[k] + (f->node_begin[t0 + k + 1] - f->node_begin[t0 + k]);
    for (int64_t k = 0; k < total; ++k) where[k] = -1;

    /* pass 1: interleaved block, level by level, trees in order */
    int64_t nf = 0;
    for (int32_t k = 0; k < nb; ++k) { frontier[nf] = 0; lvl_tree[nf] = k; ++nf; }
    for (int32_t level = 0; level <= d && nf > 0; ++level) {
        int64_t nn = 0;
        for (int32_t k = 0; k < nb; ++k) {
            for (int64_t j = 0; j < nf; ++j) {
                if (lvl_tree[j] != k) continue;
                int32_t t = t0 + k, v = frontier[j];
                int64_t b = f->node_begin[t];
                if (f->left[b + v] < 0) continue; /* leaves become class nodes */
                or_node nd = {f->feature[b + v], f->threshold[b + v], {-1, -1}, -1, v};
                int32_t me = lay_push(L, nd, t);
                if (me < 0) goto done;
                where[boff[k] + v] = me;
                next[nn] = f->left[b + v]; lvl_nodes[nn] = k; ++nn;
                next[nn] = f->right[b + v]; lvl_nodes[nn] = k; ++nn;
            }
        }
        for (int64_t j = 0; j < nn; ++j) { frontier[j] = next[j]; lvl_tree[j] = lvl_nodes[j]; }
        nf = nn;
    }
    /* pass 2: deep regions per tree, Stat order, rooted at the frontier.
     * Class nodes close the bin, so deep nodes first reference them through
     * placeholders -(c+2), patched once the class nodes exist. */
    for (int32_t c = 0; c < C; ++c) cls_node[c] = -(c + 2);
    for (int32_t k = 0; k < nb; ++k) {
        for (int64_t j = 0; j < nf; ++j) {
            if (lvl_tree[j] != k) continue;
            int32_t v = frontier[j];
            int64_t b = f->node_begin[t0 + k];
            if (f->left[b + v] < 0) continue;
            int32_t me = place_df(L, f, t0 + k, v, 1, cls_node);
            if (me < 0 && me > -2) goto done;
            where[boff[k] + v] = me;
        }
    }
    int32_t first_cls = (int32_t)L->n_nodes;
    if (append_class_nodes(L, C, -1, cls_node) < 0) goto done;
    /* patch placeholders inside deep regions */
    for (int64_t k = bin_start; k < first_cls; ++k) {
        for (int s = 0; s < 2; ++s) {
            int32_t ch = L->nodes[k].child[s];
            if (ch <= -2) L->nodes[k].child[s] = first_cls + (-ch - 2);
        }
    }
    /* link the interleaved block: children are the deep roots, interleaved
     * nodes, or class nodes */
    for (int32_t k = 0; k < nb; ++k) {
        int32_t t = t0 + k;
        int64_t b = f->node_begin[t];
        int64_t m = f->node_begin[t + 1] - b;
        for (int32_t v = 0; v < m; ++v) {
            int32_t me = where[boff[k] + v];
            if (me < 0 || f->left[b + v] < 0) continue;
            if (L->nodes[me].child[0] != -1) continue; /* deep node, already linked */
            for (int s = 0; s < 2; ++s) {
                int32_t ch = s ? f->right[b + v] : f->left[b + v];
                int32_t pos = f->left[b + ch] < 0 ? cls_node[f->leaf_class[b + ch]] : where[boff[k] + ch];
                L->nodes[me].child[s] = pos;
            }
        }
        L->root[t] = f->left[b] < 0 ? cls_node[f->leaf_class[b]] : where[boff[k] + 0];
    }
    rc = 0;
done:
    free(lvl_nodes); free(lvl_tree); free(where); free(boff); free(frontier); free(next); free(cls_node);
    return rc;
}

void or_layout_free(or_layout *L) {
    if (!L) return;
    free(L->nodes); free(L->root); free(L->tree_of); free(L);
}

/* Build one of the paper's layouts.  kind: 0 BF, 1 DF, 2 DF-, 3 Stat, 4 Bin.
 * bin_size and depth are used by Bin only.  cardinality is needed by Stat
 * and Bin.  Returns NULL on bad arguments or allocation failure. */
or_layout *or_layout_build(int32_t kind, int32_t T, int32_t C, const int64_t *node_begin, const int32_t *left,
                           const int32_t *right, const int32_t *feature, const float *threshold,
                           const int32_t *leaf_class, const int64_t *cardinality, int32_t bin_size, int32_t depth) {
    if (kind < 0 || kind > 4 || T < 1 || C < 1) return NULL;
    if (kind == OR_BIN && (bin_size < 1 || depth < 0)) return NULL;
    if ((kind == OR_STAT || kind == OR_BIN) && !cardinality) return NULL;
    or_layout *L = calloc(1, sizeof(or_layout));
    if (!L) return NULL;
    L->kind = kind; L->T = T; L->C = C; L->bin_size = bin_size; L->depth = depth;
    L->root = malloc(sizeof(int32_t) * (size_t)T);
    if (!L->root) { or_layout_free(L); return NULL; }
    forest_ref f = {node_begin, left, right, feature, leaf_class, threshold, cardinality};
    int32_t *cls_node = malloc(sizeof(int32_t) * (size_t)C);
    if (!cls_node) { or_layout_free(L); return NULL; }
    int rc = 0;
    for (int32_t t = 0; t < T && rc == 0; ) {
        if (kind == OR_BF) { rc = build_bf_tree(L, &f, t); ++t; continue; }
        if (kind == OR_DF) { int32_t r = place_df(L, &f, t, 0, 0, NULL); rc = r < 0 ? -1 : 0; L->root[t] = r; ++t; continue; }
        if (kind == OR_DFM || kind == OR_STAT) {
            /* class nodes at the end of the tree's array: place internals with
             * placeholders first, then append and patch */
            for (int32_t c = 0; c < C; ++c) cls_node[c] = -(c + 2);
            int64_t start = L->n_nodes;
            int32_t r = place_df(L, &f, t, 0, kind == OR_STAT, cls_node);
            if (r < 0 && r > -2) { rc = -1; break; }
            int32_t first_cls = (int32_t)L->n_nodes;
            if (append_class_nodes(L, C, t, cls_node) < 0) { rc = -1; break; }
            for (int64_t k = start; k < first_cls; ++k)
                for (int s = 0; s < 2; ++s)
                    if (L->nodes[k].child[s] <= -2) L->nodes[k].child[s] = first_cls + (-L->nodes[k].child[s] - 2);
            L->root[t] = r <= -2 ? first_cls + (-r - 2) : r;
            ++t;
            continue;
        }
        int32_t t1 = t + bin_size < T ? t + bin_size : T;
        rc = build_bin(L, &f, t, t1, depth, C);
        t = t1;
    }
    free(cls_node);
    if (rc != 0) { or_layout_free(L); return NULL; }
    return L;
}

int64_t or_layout_n_nodes(const or_layout *L) { return L->n_nodes; }

/* Export the layout for structural checks: per node its feature (-1 leaf or
 * class node), threshold, children, class, original tree-local id and tree. */
void or_layout_export(const or_layout *L, int32_t *feature, float *threshold, int32_t *child0, int32_t *child1,
                      int32_t *cls, int32_t *orig, int32_t *tree_of, int32_t *root) {
    for (int64_t k = 0; k < L->n_nodes; ++k) {
        const or_node *nd = &L->nodes[k];
        feature[k] = nd->feature; threshold[k] = nd->threshold;
        child0[k] = nd->child[0]; child1[k] = nd->child[1];
        cls[k] = nd->cls; orig[k] = nd->orig; tree_of[k] = L->tree_of[k];
    }
    memcpy(root, L->root, sizeof(int32_t) * (size_t)L->T);
}

/* Classify through a layout.  For each (observation, tree) reports the class
 * reached and the leaf as (tree-local id of the last internal node, direction)
 * -- the pair identifies the leaf even where leaves are merged into class
 * nodes.  A tree that is a single leaf reports (-1, 0).  Bin layouts advance
 * all trees of a bin one level per sweep (Section III-B). */
int or_layout_predict(const or_layout *L, int32_t F, const float *X, int64_t n, int32_t n_threads,
                      int32_t *out_class, int32_t *out_parent, int8_t *out_dir) {
    if (n < 0 || F < 1) return -1;
    const int32_t T = L->T;
    if (n_threads < 1) n_threads = 1;
    int bad = 0;
#pragma omp parallel for num_threads(n_threads) schedule(dynamic, 16) reduction(| : bad)
    for (int64_t i = 0; i < n; ++i) {
        const float *x = X + i * F;
        int32_t cur[4096];
        int32_t par[4096];
        int8_t dir[4096];
        const int32_t B = L->kind == OR_BIN ? L->bin_size : 1;
        if (B > 4096) { bad = 1; continue; }
        for (int32_t t0 = 0; t0 < T; t0 += B) {
            int32_t nb = t0 + B < T ? B : T - t0;
            for (int32_t k = 0; k < nb; ++k) { cur[k] = L->root[t0 + k]; par[k] = -1; dir[k] = 0; }
            int active = 1;
            while (active) { /* one sweep: every unfinished tree of the bin moves one level */
                active = 0;
                for (int32_t k = 0; k < nb; ++k) {
                    const or_node *nd = &L->nodes[cur[k]];
                    if (nd->feature < 0) continue;
                    int right = !(x[nd->feature] <= nd->threshold);
                    par[k] = nd->orig;
                    dir[k] = (int8_t)right;
                    cur[k] = nd->child[right];
                    active = 1;
                }
            }
            for (int32_t k = 0; k < nb; ++k) {
                int64_t o = i * T + t0 + k;
                out_class[o] = L->nodes[cur[k]].cls;
                out_parent[o] = par[k];
                out_dir[o] = dir[k];
            }
        }
    }
    return bad ? -1 : 0;
}

/* ------------------------------------------------------ analytic helpers */

/* Expected utility of a cache load for the Stat layout, Section III-A. */
double or_eu_stat(double bias) { return 1.0 + bias * (1.0 + bias * (1.0 + bias)); }

/* Table I quantities of a forest.  out[0] mean internal nodes per tree,
 * out[1] largest tree depth (edges from the root to the deepest leaf),
 * out[2] mean over internal nodes of max(LC, RC) / PN. */
void or_forest_stats(int32_t T, const int64_t *node_begin, const int32_t *left, const int32_t *right,
                     const int64_t *cardinality, double *out) {
    int64_t internal = 0;
    double bias_sum = 0;
    int32_t max_depth = 0;
    for (int32_t t = 0; t < T; ++t) {
        const int64_t b = node_begin[t], m = node_begin[t + 1] - b;
        if (m <= 0) continue;
        int32_t *stack = malloc(sizeof(int32_t) * (size_t)m);
        int32_t *depth = malloc(sizeof(int32_t) * (size_t)m);
        if (!stack || !depth) { free(stack); free(depth); continue; }
        int64_t sp = 0;
        stack[sp++] = 0;
        depth[0] = 0;
        while (sp > 0) { /* explicit depth-first walk from the root */
            int32_t v = stack[--sp];
            if (depth[v] > max_depth) max_depth = depth[v];
            if (left[b + v] < 0) continue;
            depth[left[b + v]] = depth[v] + 1;
            depth[right[b + v]] = depth[v] + 1;
            stack[sp++] = right[b + v];
            stack[sp++] = left[b + v];
            ++internal;
            int64_t lc = cardinality[b + left[b + v]], rc = cardinality[b + right[b + v]];
            bias_sum += (double)(lc > rc ? lc : rc) / (double)cardinality[b + v];
        }
        free(stack);
        free(depth);
    }
    out[0] = T ? (double)internal / T : 0.0;
    out[1] = max_depth;
    out[2] = internal ? bias_sum / (double)internal : 0.0;
}
