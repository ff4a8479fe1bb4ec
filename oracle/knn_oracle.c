/*
 * knn_oracle.c -- plain, slow, FP64 CPU oracle for the online k-nn graph
 * method of Debatty, Michiardi and Mees, "Fast Online k-nn Graph Building"
 * (KDD'16, arXiv 1602.06819).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: it exists so that tests, the smoke check and the CPU
 * baseline leg of the benchmark can compare the CUDA path with a plain
 * restatement of the paper.  It shares no code, header, table or constant
 * generator with the CUDA library.
 *
 * What it computes, each function citing the passage it follows:
 *   orc_exact_knn      -- brute-force exact k-nn graph (Sec. 2.1: all pairwise
 *                         similarities, keep the k best per node; it is also
 *                         the offline graph of Sec. 8.5 "Graph quality").
 *   orc_search         -- iGNNS (Sec. 3): random restarts, the expansion test
 *                         sim(q,r) < s_max/e, eager hill climbing, and the
 *                         budget of n/speedup similarity computations.
 *   orc_search_climb   -- the same search with a choice of climb: the eager
 *                         rule of iGNNS, or the GNNS rule the paper compares
 *                         against (Sec. 2.2, Sec. 3: every neighbour of the
 *                         current node is evaluated and the search moves to
 *                         the most similar one).
 *   orc_update         -- Update (Algorithm 2): walk from the found neighbours
 *                         to a fixed DEPTH and offer `new` to the lists met.
 *   orc_insert_stream  -- the sequential online build (Algorithm 1), one new
 *                         point at a time: iGNNS, then Update.
 *   orc_rescore        -- exact re-scoring of screening candidates (the
 *                         reduced-precision storage forms; the paper fixes no
 *                         precision, so the exact form is FP64 here).
 *   orc_kmedoids_*     -- balanced k-medoids (Sec. 6, Algorithm 4): the
 *                         weighted assign step with the capacity penalty
 *                         w(t, m), the medoid update, and their iteration.
 *   orc_correct_edges  -- correct edges e_c of an online graph (Sec. 8.5).
 *   orc_quality_q      -- Q = (e_c - e_u)/e_m with e_m, e_u of Sec. 8.5.
 *   orc_quantize_*     -- BF16 and FP8-E4M3 storage codes from their bit-level
 *                         definitions (screening forms only).
 *   orc_splitmix64_*   -- the counter-based generator that draws restart nodes.
 *
 * Readings where the paper is silent:
 *   similarity   sim(a,b) = 1/(1 + ||a-b||_2), computed in FP64 from the
 *                FP32 values given.  Higher is closer.
 *   order        entry x is better than y iff sim_x > sim_y, or the sims are
 *                equal and id_x < id_y.  Every list is sorted best first.
 *   budget       B = max(1, floor(n / speedup)); every similarity computed
 *                by the search counts, discarded restarts included.
 *   expansion    s_max starts at -inf, so the first restart is always kept;
 *                a restart is discarded iff sim < s_max / e (strict); e <= 0
 *                or e = inf disables discarding.
 *   visited      no node's similarity is computed twice within one search;
 *                drawing a visited or removed node is a free redraw; at most
 *                64*n draws, and the search stops when every live node has
 *                been visited.
 *   draws        the j-th restart draw of a search is
 *                  r_j = floor(x_j * n / 2^64),
 *                  x_j = SplitMix64 output j of the generator seeded with
 *                        h = mix(seed XOR mix(stream)),
 *                with mix(v) the first output of SplitMix64 seeded with v
 *                (Steele, Lea and Flood, OOPSLA 2014) and the range
 *                reduction the multiply-shift of Lemire (2019).
 *   climb        neighbours of cur are scanned in stored (best-first) order;
 *                the first one whose similarity is strictly greater than
 *                sim(q, cur) becomes cur and the scan starts again.
 *   GNNS climb   every unvisited neighbour of cur is evaluated (in stored
 *                order, until the budget is spent); the most similar of
 *                them (ties to the earlier position) becomes cur when it is
 *                strictly more similar than cur.  Visited neighbours are
 *                skipped as in iGNNS (no similarity is computed twice), and
 *                the search runs on the same budget and restart draws, so
 *                the two rules compare at equal evaluations.  Hajebi et
 *                al.'s fixed restart count and depth cap are replaced by
 *                that budget, and GNNS runs without the expansion test
 *                (e = inf).
 *   update       level-1 sims are the ones the search returned (not counted
 *                again); lists are read before `new` is offered to them;
 *                the next level is the distinct ids gathered, minus nodes
 *                already seen, minus `new`, minus removed nodes.
 *   offer        the new node enters a list when its id is absent and the
 *                list has a free slot or the candidate is better than its
 *                last entry: it is placed in sorted position and the entry
 *                pushed past k drops out.
 *
 * Decision margins: every floating-point decision records its relative
 * margin, so that a test can tell a genuine mismatch from a near tie that
 * FP32 rounding on the GPU may legitimately decide the other way.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Similarity (Sec. 3 uses any similarity; the synthetic data uses L2).      */
/* ------------------------------------------------------------------------- */

static double squared_l2(const float *a, const float *b, int32_t d)
{
    double acc = 0.0;
    for (int32_t i = 0; i < d; ++i) {
        double diff = (double)a[i] - (double)b[i];
        acc += diff * diff;
    }
    return acc;
}

static double similarity(const float *a, const float *b, int32_t d)
{
    return 1.0 / (1.0 + sqrt(squared_l2(a, b, d)));
}

double orc_similarity(const float *a, const float *b, int32_t d)
{
    return similarity(a, b, d);
}

/* better(x, y): higher similarity first, lower id on equal similarity. */
static int better(double sim_x, int64_t id_x, double sim_y, int64_t id_y)
{
    return sim_x > sim_y || (sim_x == sim_y && id_x < id_y);
}

static double rel_gap(double a, double b)
{
    double m = fabs(a) > fabs(b) ? fabs(a) : fabs(b);
    if (m == 0.0) return 0.0;
    return fabs(a - b) / m;
}

/* Margin of a comparison between two similarities.  Exactly equal values
 * (duplicate points) are no hazard: both sides compute them equal and break
 * the tie by id, so they count as an infinite margin. */
static double sim_gap(double a, double b)
{
    return a == b ? INFINITY : rel_gap(a, b);
}

/* ------------------------------------------------------------------------- */
/* SplitMix64 (Steele, Lea, Flood 2014) and the restart draw.                */
/* ------------------------------------------------------------------------- */

static const uint64_t SPLITMIX_GAMMA = 0x9E3779B97F4A7C15ULL;

static uint64_t splitmix_finalize(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Output number j (0-based) of a SplitMix64 generator whose state starts at
 * `seed`: the state is advanced by the golden gamma before each output. */
uint64_t orc_splitmix64_output(uint64_t seed, uint64_t j)
{
    return splitmix_finalize(seed + (j + 1) * SPLITMIX_GAMMA);
}

static uint64_t mix(uint64_t v) { return orc_splitmix64_output(v, 0); }

uint64_t orc_search_key(uint64_t seed, uint64_t stream)
{
    return mix(seed ^ mix(stream));
}

/* Node drawn by restart draw j of the search keyed by `key`, among n nodes. */
int64_t orc_draw(uint64_t key, uint64_t j, int64_t n)
{
    uint64_t x = orc_splitmix64_output(key, j);
    unsigned __int128 p = (unsigned __int128)x * (unsigned __int128)(uint64_t)n;
    return (int64_t)(uint64_t)(p >> 64);
}

/* ------------------------------------------------------------------------- */
/* A bounded, sorted result list (the "set of the most similar points").      */
/* ------------------------------------------------------------------------- */

typedef struct {
    int32_t cap;      /* entries kept                                      */
    int32_t len;
    int64_t *ids;
    double *sims;
} best_list;

static void best_list_offer(best_list *b, double s, int64_t id)
{
    if (b->len == b->cap && !better(s, id, b->sims[b->len - 1], b->ids[b->len - 1]))
        return;
    int32_t pos = b->len < b->cap ? b->len : b->cap - 1;
    while (pos > 0 && better(s, id, b->sims[pos - 1], b->ids[pos - 1])) {
        b->sims[pos] = b->sims[pos - 1];
        b->ids[pos] = b->ids[pos - 1];
        --pos;
    }
    b->sims[pos] = s;
    b->ids[pos] = id;
    if (b->len < b->cap) ++b->len;
}

/* Smallest relative gap between consecutive entries of the first `upto`+1
 * entries: a near tie there can reorder or swap the boundary entry. */
static double best_list_margin(const best_list *b, int32_t upto)
{
    double m = INFINITY;
    int32_t last = upto < b->len - 1 ? upto : b->len - 1;
    for (int32_t i = 0; i < last; ++i) {
        double g = sim_gap(b->sims[i], b->sims[i + 1]);
        if (g < m) m = g;
    }
    return m;
}

/* ------------------------------------------------------------------------- */
/* Exact k-nn graph by brute force (Sec. 2.1; the offline graph of Sec. 8.5) */
/* ------------------------------------------------------------------------- */

/* For each requested row u: the k live nodes v != u most similar to u.
 * rows == NULL means every row 0..n-1.  out_margin[r] is the smallest
 * relative gap among the k+1 best (near ties that FP32 may order
 * differently).  Missing entries are id -1 and sim -inf. */
void orc_exact_knn(const float *X, int64_t n, int32_t d, int32_t k,
                   const int64_t *rows, int64_t n_rows, const uint8_t *removed,
                   int64_t *out_ids, double *out_sims, double *out_margin)
{
    if (rows == NULL) n_rows = n;
#pragma omp parallel
    {
        best_list b;
        b.cap = k + 1;
        b.ids = (int64_t *)malloc(sizeof(int64_t) * (size_t)(k + 1));
        b.sims = (double *)malloc(sizeof(double) * (size_t)(k + 1));
#pragma omp for schedule(dynamic, 16)
        for (int64_t r = 0; r < n_rows; ++r) {
            int64_t u = rows ? rows[r] : r;
            b.len = 0;
            for (int64_t v = 0; v < n; ++v) {
                if (v == u || (removed && removed[v])) continue;
                best_list_offer(&b, similarity(X + u * d, X + v * d, d), v);
            }
            for (int32_t i = 0; i < k; ++i) {
                out_ids[r * k + i] = i < b.len ? b.ids[i] : -1;
                out_sims[r * k + i] = i < b.len ? b.sims[i] : -INFINITY;
            }
            if (out_margin) out_margin[r] = best_list_margin(&b, k);
        }
        free(b.ids);
        free(b.sims);
    }
}

/* ------------------------------------------------------------------------- */
/* iGNNS (Sec. 3).                                                           */
/* ------------------------------------------------------------------------- */

typedef struct {
    int64_t evals;      /* similarities computed (the budget counter)          */
    int64_t budget;     /* B = max(1, floor(n/speedup))                        */
    int64_t restarts;   /* random nodes evaluated                              */
    int64_t discarded;  /* of which discarded by the expansion test            */
    int64_t moves;      /* eager moves to a more similar neighbour             */
    int64_t draws;      /* draws made, free redraws included                   */
    double min_margin;  /* smallest relative margin of any decision            */
} orc_search_stats;

enum { ORC_CLIMB_EAGER = 0, ORC_CLIMB_BEST = 1 };

static void note_margin(orc_search_stats *st, double m)
{
    if (m < st->min_margin) st->min_margin = m;
}

/*
 * Search the graph (X: n rows of d floats; nbr_ids: n rows of k ids, best
 * first, -1 for an empty slot) for the k_out nodes most similar to q.
 *
 * draws/n_draws: when draws != NULL the restart nodes are taken from this
 * list in order instead of the generator (hand-traced tests); the search
 * ends when the list is exhausted.
 *
 * Returns the number of results written (<= k_out), best first.
 */
int32_t orc_search_climb(const float *X, int64_t n, int32_t d,
                         const int64_t *nbr_ids, int32_t k, const uint8_t *removed,
                         const float *q, int32_t k_out,
                         double speedup, double expansion, uint64_t seed, uint64_t stream,
                         const int64_t *draws, int64_t n_draws, int32_t climb,
                         int64_t *out_ids, double *out_sims, orc_search_stats *st);

int32_t orc_search(const float *X, int64_t n, int32_t d,
                   const int64_t *nbr_ids, int32_t k, const uint8_t *removed,
                   const float *q, int32_t k_out,
                   double speedup, double expansion, uint64_t seed, uint64_t stream,
                   const int64_t *draws, int64_t n_draws,
                   int64_t *out_ids, double *out_sims, orc_search_stats *st)
{
    return orc_search_climb(X, n, d, nbr_ids, k, removed, q, k_out, speedup, expansion, seed,
                            stream, draws, n_draws, ORC_CLIMB_EAGER, out_ids, out_sims, st);
}

/* climb: ORC_CLIMB_EAGER (iGNNS) or ORC_CLIMB_BEST (GNNS). */
int32_t orc_search_climb(const float *X, int64_t n, int32_t d,
                         const int64_t *nbr_ids, int32_t k, const uint8_t *removed,
                         const float *q, int32_t k_out,
                         double speedup, double expansion, uint64_t seed, uint64_t stream,
                         const int64_t *draws, int64_t n_draws, int32_t climb,
                         int64_t *out_ids, double *out_sims, orc_search_stats *st)
{
    memset(st, 0, sizeof(*st));
    st->min_margin = INFINITY;

    int64_t B = (int64_t)floor((double)n / speedup);   /* "n / speedup" */
    if (B < 1) B = 1;
    st->budget = B;
    int discard_enabled = expansion > 0.0 && isfinite(expansion);

    int64_t n_live = 0;
    for (int64_t v = 0; v < n; ++v) n_live += !(removed && removed[v]);

    uint8_t *visited = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    int64_t n_visited = 0;

    best_list topk;
    topk.cap = k_out + 1;          /* one extra entry to measure the boundary */
    topk.len = 0;
    topk.ids = (int64_t *)malloc(sizeof(int64_t) * (size_t)(k_out + 1));
    topk.sims = (double *)malloc(sizeof(double) * (size_t)(k_out + 1));

    double s_max = -INFINITY;
    uint64_t key = orc_search_key(seed, stream);
    uint64_t j = 0;
    const uint64_t max_draws = 64ULL * (uint64_t)(n > 0 ? n : 1);
    int out_of_budget = 0;

    while (!out_of_budget && st->evals < B && n_visited < n_live) {
        /* restart with a random node r */
        int64_t r;
        if (draws) {
            if ((int64_t)j >= n_draws) break;
            r = draws[j++];
        } else {
            if (j >= max_draws) break;
            r = orc_draw(key, j++, n);
        }
        st->draws++;
        if (visited[r] || (removed && removed[r])) continue;   /* free redraw */

        double s = similarity(q, X + r * d, d);
        st->evals++;
        st->restarts++;
        visited[r] = 1;
        n_visited++;
        best_list_offer(&topk, s, r);

        /* expansion test: discard r if sim(q, r) < s_max / e */
        if (discard_enabled && s_max > -INFINITY) {
            double threshold = s_max / expansion;
            note_margin(st, rel_gap(s, threshold));
            if (s < threshold) {
                st->discarded++;
                continue;
            }
        }
        if (s > s_max) s_max = s;

        int64_t cur = r;
        double s_cur = s;
        int moved = 1;
        /* GNNS hill climbing from r: evaluate every unvisited neighbour,
         * then move to the most similar one if it beats cur */
        while (climb == ORC_CLIMB_BEST && moved && !out_of_budget) {
            moved = 0;
            int64_t best = -1;
            double s_best = -INFINITY;
            for (int32_t i = 0; i < k; ++i) {
                int64_t nb = nbr_ids[cur * k + i];
                if (nb < 0 || visited[nb] || (removed && removed[nb])) continue;
                if (st->evals == B) { out_of_budget = 1; break; }
                double s_nb = similarity(q, X + nb * d, d);
                st->evals++;
                visited[nb] = 1;
                n_visited++;
                best_list_offer(&topk, s_nb, nb);
                if (s_nb > s_max) s_max = s_nb;
                if (best >= 0) note_margin(st, sim_gap(s_nb, s_best));
                if (s_nb > s_best) {     /* ties keep the earlier position */
                    best = nb;
                    s_best = s_nb;
                }
            }
            if (best < 0) break;         /* every neighbour visited: local maximum */
            note_margin(st, sim_gap(s_best, s_cur));
            if (s_best > s_cur) {
                cur = best;
                s_cur = s_best;
                st->moves++;
                moved = 1;
            }
        }
        /* eager hill climbing from r */
        while (climb == ORC_CLIMB_EAGER && moved && !out_of_budget) {
            moved = 0;
            for (int32_t i = 0; i < k; ++i) {
                int64_t nb = nbr_ids[cur * k + i];
                if (nb < 0 || visited[nb] || (removed && removed[nb])) continue;
                if (st->evals == B) { out_of_budget = 1; break; }
                double s_nb = similarity(q, X + nb * d, d);
                st->evals++;
                visited[nb] = 1;
                n_visited++;
                best_list_offer(&topk, s_nb, nb);
                if (s_nb > s_max) s_max = s_nb;
                note_margin(st, sim_gap(s_nb, s_cur));
                if (s_nb > s_cur) {          /* first increase: move there */
                    cur = nb;
                    s_cur = s_nb;
                    st->moves++;
                    moved = 1;
                    break;
                }
            }
        }
    }

    int32_t found = topk.len < k_out ? topk.len : k_out;
    for (int32_t i = 0; i < k_out; ++i) {
        out_ids[i] = i < found ? topk.ids[i] : -1;
        out_sims[i] = i < found ? topk.sims[i] : -INFINITY;
    }
    note_margin(st, best_list_margin(&topk, k_out));
    free(visited);
    free(topk.ids);
    free(topk.sims);
    return found;
}

/* Exact re-score of screening candidates: the similarity of q to each
 * candidate from the exact vectors, keeping the k_out best.  The margin is
 * the smallest relative gap among the k_out+1 best re-scored entries. */
int32_t orc_rescore(const float *X, int32_t d, const float *q,
                    const int64_t *cand_ids, int32_t n_cand, int32_t k_out,
                    int64_t *out_ids, double *out_sims, double *out_margin)
{
    best_list b;
    b.cap = k_out + 1;
    b.len = 0;
    b.ids = (int64_t *)malloc(sizeof(int64_t) * (size_t)(k_out + 1));
    b.sims = (double *)malloc(sizeof(double) * (size_t)(k_out + 1));
    for (int32_t c = 0; c < n_cand; ++c) {
        if (cand_ids[c] < 0) continue;
        best_list_offer(&b, similarity(q, X + cand_ids[c] * d, d), cand_ids[c]);
    }
    int32_t found = b.len < k_out ? b.len : k_out;
    for (int32_t i = 0; i < k_out; ++i) {
        out_ids[i] = i < found ? b.ids[i] : -1;
        out_sims[i] = i < found ? b.sims[i] : -INFINITY;
    }
    if (out_margin) *out_margin = best_list_margin(&b, k_out);
    free(b.ids);
    free(b.sims);
    return found;
}

/* ------------------------------------------------------------------------- */
/* Update (Algorithm 2).                                                     */
/* ------------------------------------------------------------------------- */

typedef struct {
    int64_t evals;          /* similarities computed by the update (levels >= 2) */
    int64_t literal_evals;  /* Algorithm 2's own count: every node popped        */
    int64_t offers_taken;   /* lists that received `new`                         */
    double min_margin;      /* smallest relative gap between `new` and an entry  */
} orc_update_stats;

/* The offer rule of Update (Algorithm 2): `id` joins the list when it is not
 * in it yet and the list has a free slot or `id` ranks above the last entry;
 * the entry pushed past k drops out.  Returns 1 if the list changed.  The
 * margin is the smallest relative gap between s and any entry of the list
 * (a near tie there may place `id` differently). */
static int offer_to_list(int64_t *ids, double *sims, int32_t k, double s, int64_t id,
                         double *margin)
{
    int32_t len = 0;
    while (len < k && ids[len] >= 0) {
        if (ids[len] == id) return 0;
        ++len;
    }
    for (int32_t i = 0; i < len; ++i) {
        double g = sim_gap(s, sims[i]);
        if (g < *margin) *margin = g;
    }
    if (len == k && !better(s, id, sims[k - 1], ids[k - 1])) return 0;
    int32_t pos = len < k ? len : k - 1;
    while (pos > 0 && better(s, id, sims[pos - 1], ids[pos - 1])) {
        sims[pos] = sims[pos - 1];
        ids[pos] = ids[pos - 1];
        --pos;
    }
    sims[pos] = s;
    ids[pos] = id;
    return 1;
}

static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

/*
 * Update (Algorithm 2) for a new node already stored at row new_id of X,
 * whose own list the caller has set: a breadth-first walk of at most `depth`
 * levels that starts at the neighbours the search found and offers the new
 * node to the list of every node it reaches.  L_ids/L_sims: the search's
 * result, best first (L_len entries).
 *
 * full != 0 replaces the walk by an offer to every live node (used only to
 * check the offer rule against brute force).
 */
void orc_update(const float *X, int64_t n_total, int32_t d,
                int64_t *nbr_ids, double *nbr_sims, int32_t k,
                const uint8_t *removed, int64_t new_id,
                const int64_t *L_ids, const double *L_sims, int32_t L_len,
                int32_t depth, int32_t full, orc_update_stats *st)
{
    memset(st, 0, sizeof(*st));
    st->min_margin = INFINITY;
    const float *x_new = X + new_id * d;

    if (full) {
        for (int64_t w = 0; w < n_total; ++w) {
            if (w == new_id || (removed && removed[w])) continue;
            double s = similarity(x_new, X + w * d, d);
            st->evals++;
            st->literal_evals++;
            st->offers_taken += offer_to_list(nbr_ids + w * k, nbr_sims + w * k, k, s,
                                              new_id, &st->min_margin);
        }
        return;
    }

    uint8_t *seen = (uint8_t *)calloc((size_t)n_total, 1);
    seen[new_id] = 1;

    /* level 1: the nodes of the search result, with the search's similarities */
    int64_t lv_len = 0, lv_cap = L_len > 0 ? L_len : 1;
    int64_t *lv_ids = (int64_t *)malloc(sizeof(int64_t) * (size_t)lv_cap);
    double *lv_sims = (double *)malloc(sizeof(double) * (size_t)lv_cap);
    for (int32_t i = 0; i < L_len; ++i) {
        if (L_ids[i] < 0 || seen[L_ids[i]]) continue;
        seen[L_ids[i]] = 1;
        lv_ids[lv_len] = L_ids[i];
        lv_sims[lv_len] = L_sims[i];
        ++lv_len;
    }

    for (int32_t level = 1; level <= depth && lv_len > 0; ++level) {
        int64_t got = 0, got_cap = lv_len * k;
        int64_t *gathered = (int64_t *)malloc(sizeof(int64_t) * (size_t)(got_cap > 0 ? got_cap : 1));
        for (int64_t li = 0; li < lv_len; ++li) {
            int64_t node = lv_ids[li];
            int64_t *list_ids = nbr_ids + node * k;
            double *list_sims = nbr_sims + node * k;
            /* the node's list feeds the next level; it is read before the
             * new node is offered to it */
            if (level < depth)
                for (int32_t i = 0; i < k; ++i)
                    if (list_ids[i] >= 0) gathered[got++] = list_ids[i];
            /* level 1 takes the search's similarity, deeper levels compute it */
            double s;
            if (level == 1) {
                s = lv_sims[li];
            } else {
                s = similarity(x_new, X + node * d, d);
                st->evals++;
            }
            st->literal_evals++;
            st->offers_taken += offer_to_list(list_ids, list_sims, k, s, new_id,
                                              &st->min_margin);
        }
        /* the next level: each gathered id once, in ascending order, leaving
         * out nodes already seen (the new node among them) and removed ones */
        qsort(gathered, (size_t)got, sizeof(int64_t), cmp_i64);
        free(lv_ids);
        free(lv_sims);
        lv_cap = got > 0 ? got : 1;
        lv_ids = (int64_t *)malloc(sizeof(int64_t) * (size_t)lv_cap);
        lv_sims = (double *)malloc(sizeof(double) * (size_t)lv_cap);
        lv_len = 0;
        for (int64_t i = 0; i < got; ++i) {
            int64_t w = gathered[i];
            if (seen[w] || (removed && removed[w])) continue;
            seen[w] = 1;
            lv_ids[lv_len] = w;
            lv_sims[lv_len] = NAN;
            ++lv_len;
        }
        free(gathered);
    }
    free(lv_ids);
    free(lv_sims);
    free(seen);
}

/* ------------------------------------------------------------------------- */
/* Sequential online build (Algorithm 1).                                     */
/* ------------------------------------------------------------------------- */

typedef struct {
    int64_t search_evals;
    int64_t update_evals;
    int64_t update_literal_evals;
    double search_margin;
    double update_margin;
} orc_insert_stats;

/*
 * Add the m points stored at rows n0 .. n0+m-1 of X to the graph whose first
 * n0 rows are built, one at a time: each point is searched with iGNNS, its
 * list is the result, and Update then walks from that result.  The search
 * of point i sees n0+i nodes and uses stream = its id.  nbr_ids/nbr_sims
 * have room for n0+m rows.
 */
void orc_insert_stream(const float *X, int64_t n0, int64_t m, int32_t d,
                       int64_t *nbr_ids, double *nbr_sims, int32_t k,
                       const uint8_t *removed,
                       double speedup, double expansion, int32_t depth, uint64_t seed,
                       orc_insert_stats *stats)
{
    orc_search_stats ss;
    orc_update_stats us;
    for (int64_t i = 0; i < m; ++i) {
        int64_t new_id = n0 + i;
        int64_t *L_ids = nbr_ids + new_id * k;
        double *L_sims = nbr_sims + new_id * k;
        /* Search: the current graph holds nodes 0 .. new_id-1 */
        orc_search(X, new_id, d, nbr_ids, k, removed, X + new_id * d, k,
                   speedup, expansion, seed, (uint64_t)new_id, NULL, 0,
                   L_ids, L_sims, &ss);
        /* Update: the new node joins the graph with the list found */
        orc_update(X, new_id + 1, d, nbr_ids, nbr_sims, k, removed, new_id,
                   L_ids, L_sims, k, depth, 0, &us);
        if (stats) {
            stats[i].search_evals = ss.evals;
            stats[i].update_evals = us.evals;
            stats[i].update_literal_evals = us.literal_evals;
            stats[i].search_margin = ss.min_margin;
            stats[i].update_margin = us.min_margin;
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Graph quality (Sec. 8.5, "Graph quality").                                */
/* ------------------------------------------------------------------------- */

/* Number of directed edges u->v present in both graphs (n rows of k ids). */
int64_t orc_correct_edges(const int64_t *ids_a, const int64_t *ids_b, int64_t n, int32_t k)
{
    int64_t c = 0;
    for (int64_t u = 0; u < n; ++u)
        for (int32_t i = 0; i < k; ++i) {
            int64_t v = ids_a[u * k + i];
            if (v < 0) continue;
            for (int32_t j = 0; j < k; ++j)
                if (ids_b[u * k + j] == v) { ++c; break; }
        }
    return c;
}

/* e_m = n_a k + n k n_a/(n_a+n);  e_u = (n+n_a)k - e_m;  Q = (e_c - e_u)/e_m */
double orc_quality_q(int64_t e_c, int64_t n, int64_t n_a, int32_t k)
{
    double e_m = (double)n_a * k + (double)n * k * (double)n_a / (double)(n_a + n);
    double e_u = (double)(n + n_a) * k - e_m;
    return ((double)e_c - e_u) / e_m;
}

/* ------------------------------------------------------------------------- */
/* Storage codes for the screening forms.                                    */
/* ------------------------------------------------------------------------- */

static uint32_t f32_bits(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }
static float bits_f32(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }

/* bfloat16 = the upper 16 bits of an IEEE binary32, rounded to nearest even. */
uint16_t orc_bf16_code(float f)
{
    uint32_t u = f32_bits(f);
    if ((u & 0x7F800000u) == 0x7F800000u && (u & 0x007FFFFFu))
        return (uint16_t)((u >> 16) | 0x40u);             /* quiet NaN */
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7FFFu + lsb;
    return (uint16_t)(u >> 16);
}

float orc_bf16_value(uint16_t code) { return bits_f32((uint32_t)code << 16); }

/* OCP FP8 E4M3 ("fn": no infinities): 1 sign bit, 4 exponent bits with bias
 * 7, 3 mantissa bits; largest finite magnitude 448; subnormal step 2^-9.
 * Round to nearest even, saturating finite values to +-448. */
uint8_t orc_e4m3_code(float f)
{
    double a = fabs((double)f);
    uint8_t sign = (f32_bits(f) >> 31) ? 0x80u : 0x00u;
    if (isnan(a)) return (uint8_t)(sign | 0x7Fu);
    if (a >= 448.0) return (uint8_t)(sign | 0x7Eu);        /* 1.75 * 2^8 */
    int e;
    frexp(a, &e);                        /* a = f * 2^e, f in [0.5, 1) */
    int unbiased = e - 1;                /* a in [2^unbiased, 2^(unbiased+1)) */
    if (unbiased < -6) unbiased = -6;    /* subnormal range shares 2^-6's step */
    double quantum = ldexp(1.0, unbiased - 3);
    double units = nearbyint(a / quantum);   /* exact scaling, then RNE */
    double v = units * quantum;
    if (v == 0.0) return sign;
    int ve;
    frexp(v, &ve);
    int exp_field = (ve - 1) + 7;
    uint8_t bits;
    if (exp_field <= 0) {                /* subnormal: v = m * 2^-9 */
        bits = (uint8_t)(int)(v / ldexp(1.0, -9));
    } else {
        double mant = v / ldexp(1.0, ve - 1) - 1.0;       /* in [0, 1) */
        bits = (uint8_t)((exp_field << 3) | (int)(mant * 8.0));
    }
    return (uint8_t)(sign | bits);
}

float orc_e4m3_value(uint8_t code)
{
    int s = code >> 7, ef = (code >> 3) & 0xF, mf = code & 7;
    double v;
    if (ef == 0xF && mf == 7) return NAN;
    if (ef == 0) v = ldexp((double)mf, -9);
    else v = ldexp(1.0 + mf / 8.0, ef - 7);
    return (float)(s ? -v : v);
}

/* BF16 storage: code and dequantized value of every element. */
void orc_quantize_bf16(const float *X, int64_t count, uint16_t *codes, float *deq)
{
    for (int64_t i = 0; i < count; ++i) {
        codes[i] = orc_bf16_code(X[i]);
        deq[i] = orc_bf16_value(codes[i]);
    }
}

/* FP8-E4M3 storage with a per-row scale: scale = amax/448 in binary32;
 * code = e4m3(x / scale) (binary32 division); dequantized value =
 * binary32(e4m3 value * scale).  An all-zero row gets scale 1. */
void orc_quantize_e4m3(const float *X, int64_t n, int32_t d,
                       uint8_t *codes, float *scales, float *deq)
{
    for (int64_t r = 0; r < n; ++r) {
        const float *x = X + r * d;
        float amax = 0.0f;
        for (int32_t i = 0; i < d; ++i) {
            float a = fabsf(x[i]);
            if (a > amax) amax = a;
        }
        volatile float scale = amax > 0.0f ? amax / 448.0f : 1.0f;
        scales[r] = scale;
        for (int32_t i = 0; i < d; ++i) {
            volatile float v = x[i] / scale;
            uint8_t c = orc_e4m3_code(v);
            codes[r * d + i] = c;
            volatile float back = orc_e4m3_value(c) * scale;
            deq[r * d + i] = back;
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Balanced k-medoids (Sec. 6, Algorithm 4).                                 */
/*                                                                           */
/* The paper partitions a graph for its distributed search with a balanced   */
/* k-medoids clustering: p initial medoids drawn at random; the data spread */
/* over c compute nodes; each compute node assigns its points, one after    */
/* the other, to the medoid m that maximises sim(m, x) * w(t, m) with        */
/*   w(t, m) = 1 - |C_t(m)| / capacity,  capacity = n * imbalance / (p * c), */
/* |C_t(m)| counting the points that compute node has given m so far; then  */
/* every cluster takes as new medoid the member with the smallest sum of     */
/* distances to the other members, and the two steps repeat.                */
/*                                                                           */
/* Readings: the c "compute nodes" are c chunks of consecutive ids,          */
/* chunk j = [floor(j n / c), floor((j+1) n / c)) (the input order of the   */
/* synthetic data is random, so this is a random split), each assigned in   */
/* id order; the clusters are ordered by medoid position and an argmax tie  */
/* goes to the lower position; the distance of the update step is the       */
/* Euclidean distance (the paper's Spark version measures shortest paths in */
/* the graph there, and the Euclidean similarity in the assign step); an    */
/* empty cluster keeps its medoid; an update tie goes to the lower id.      */
/* The initial medoids are the first p distinct nodes drawn with the        */
/* restart generator keyed (seed, stream 2^62).                             */
/* ------------------------------------------------------------------------- */

#define ORC_KMEDOIDS_STREAM (1ULL << 62)

/* p distinct initial medoids (p <= n). */
void orc_kmedoids_init(int64_t n, int32_t p, uint64_t seed, int64_t *medoids)
{
    uint64_t key = orc_search_key(seed, ORC_KMEDOIDS_STREAM);
    uint8_t *taken = (uint8_t *)calloc((size_t)n, 1);
    int32_t got = 0;
    for (uint64_t j = 0; got < p; ++j) {
        int64_t r = orc_draw(key, j, n);
        if (taken[r]) continue;
        taken[r] = 1;
        medoids[got++] = r;
    }
    free(taken);
}

/* Assign step.  labels[i] = cluster (medoid position) of node i; margins[i]
 * (nullable) = relative gap between the best and second-best weighted
 * similarity of that decision. */
void orc_kmedoids_assign(const float *X, int64_t n, int32_t d, const int64_t *medoids, int32_t p,
                         double imbalance, int32_t chunks, int32_t *labels, double *margins)
{
    double capacity = (double)n * imbalance / ((double)p * (double)chunks);
    int64_t *count = (int64_t *)malloc(sizeof(int64_t) * (size_t)p);
    for (int32_t c = 0; c < chunks; ++c) {
        int64_t lo = (int64_t)(((__int128)c * n) / chunks);
        int64_t hi = (int64_t)(((__int128)(c + 1) * n) / chunks);
        for (int32_t m = 0; m < p; ++m) count[m] = 0;
        for (int64_t i = lo; i < hi; ++i) {
            int32_t best = -1;
            double s_best = -INFINITY, s_second = -INFINITY;
            for (int32_t m = 0; m < p; ++m) {
                double w = 1.0 - (double)count[m] / capacity;
                double score = similarity(X + i * d, X + medoids[m] * d, d) * w;
                if (score > s_best) {
                    s_second = s_best;
                    s_best = score;
                    best = m;
                } else if (score > s_second) {
                    s_second = score;
                }
            }
            labels[i] = best;
            count[best]++;
            if (margins) margins[i] = p > 1 ? rel_gap(s_best, s_second) : INFINITY;
        }
    }
    free(count);
}

/* Update step for one cluster: the member (ids `members`, cnt >= 1) whose sum
 * of Euclidean distances to the other members is smallest, ties to the lower
 * id; *margin = relative gap to the runner-up (inf for one member). */
int64_t orc_kmedoids_medoid(const float *X, int32_t d, const int64_t *members, int64_t cnt,
                            double *margin)
{
    int64_t best = -1;
    double s_best = INFINITY, s_second = INFINITY;
    for (int64_t a = 0; a < cnt; ++a) {
        double sum = 0.0;
        for (int64_t b = 0; b < cnt; ++b)
            sum += sqrt(squared_l2(X + members[a] * d, X + members[b] * d, d));
        int64_t id = members[a];
        if (sum < s_best || (sum == s_best && id < best)) {
            s_second = s_best;
            s_best = sum;
            best = id;
        } else if (sum < s_second) {
            s_second = sum;
        }
    }
    if (margin) *margin = cnt > 1 ? rel_gap(s_best, s_second) : INFINITY;
    return best;
}

/* Algorithm 4: `iters` rounds of (assign, update), then a final assign.
 * labels [n]; medoids [p] (those of the final assign); *min_margin = the
 * smallest decision margin of the whole run. */
void orc_kmedoids(const float *X, int64_t n, int32_t d, int32_t p, double imbalance,
                  int32_t chunks, int32_t iters, uint64_t seed, int32_t *labels, int64_t *medoids,
                  double *min_margin)
{
    double *margins = (double *)malloc(sizeof(double) * (size_t)n);
    int64_t *members = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    double mm = INFINITY;
    orc_kmedoids_init(n, p, seed, medoids);
    for (int32_t it = 0; ; ++it) {
        orc_kmedoids_assign(X, n, d, medoids, p, imbalance, chunks, labels, margins);
        for (int64_t i = 0; i < n; ++i)
            if (margins[i] < mm) mm = margins[i];
        if (it == iters) break;
        for (int32_t m = 0; m < p; ++m) {
            int64_t cnt = 0;
            for (int64_t i = 0; i < n; ++i)
                if (labels[i] == m) members[cnt++] = i;
            if (cnt == 0) continue;
            double g;
            medoids[m] = orc_kmedoids_medoid(X, d, members, cnt, &g);
            if (g < mm) mm = g;
        }
    }
    if (min_margin) *min_margin = mm;
    free(margins);
    free(members);
}
