/*
 * FP64 CPU oracle for batched move evaluation in stochastic open-pit scheduling.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's
 * CPU-baseline leg may load this library.  It shares no code, header, table or
 * constant with the CUDA library; the two only consume the same seeded inputs.
 *
 * Everything is plain IEEE double arithmetic (built with -ffp-contract=off),
 * written to be checked against the paper by eye:
 *
 *   - Objective (Section 5.6, Eq. 14): scenario-averaged, discounted value of
 *     the blocks mined in each period.  The second stage (Eq. 17-21) is read as
 *     a single processing mode: a block is ore in scenario s when processing it
 *     is worth more than sending it to the dump (Eq. 18: a zero processed mass
 *     means waste), and the mill's ore tonnage per period is held to a target
 *     by piecewise-linear shortfall/excess penalties.  Cash flows, penalties
 *     included, are discounted per period (Section 7.1.2).
 *   - Precedence (Eq. 15): every direct predecessor is mined in the same or an
 *     earlier period.  Capacity (Eq. 16): mined tonnage per period <= M_t.
 *   - Discount d_t = (1+r)^-t with t counted from 0 (Algorithm 5 discounts
 *     period t by 1/1.08^t).  An unmined block has period value T and d_T = 0.
 *
 * Move semantics (the candidates of Algorithm 5 / the assignment step of
 * Algorithm 4): a shift moves one block to a new period; a swap exchanges the
 * periods of two blocks.  The brute-force evaluator applies the move to a copy
 * of the schedule and recomputes every scenario's NPV from scratch: that is the
 * definition of the move's NPV delta.  The incremental evaluator is a second,
 * independently written O(S)-per-move evaluator, checked against brute force.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t B, S, T;
    const int32_t *pred_ptr; /* [B+1] CSR offsets of direct predecessors */
    const int32_t *pred_idx; /* [E]   predecessor block ids */
    const uint32_t *mass;    /* [B] tonnes */
    const double *grade;     /* [B*S] g/t, scenario fastest */
    const uint64_t *cap;     /* [T] tonnes, mining capacity M_t */
    const uint64_t *target;  /* [T] tonnes, mill ore target Q_t */
    double price, recovery, mining_cost, proc_cost;
    double shortfall_pen, excess_pen, discount_rate, lambda;
    const double *sigma;     /* [T*S] uncertainty weights sigma(s,t), period-major; NULL = none */
} or_model;

/* ------------------------------------------------------------------ setup */

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Direct predecessors of the 1-5 pattern on an nx*ny*nz grid (z = 0 on top):
 * the block straight above and its four edge neighbours on the level above,
 * clipped at the grid boundary.  b = x + nx*(y + ny*z).  Returns the arc
 * count; fills ptr[B+1] and idx[E] when they are non-NULL. */
int64_t or_stencil_preds(int32_t nx, int32_t ny, int32_t nz, int32_t *ptr, int32_t *idx) {
    int64_t e = 0;
    int32_t B = nx * ny * nz;
    for (int32_t b = 0; b < B; b++) {
        int32_t x = b % nx, y = (b / nx) % ny, z = b / (nx * ny);
        if (ptr) ptr[b] = (int32_t)e;
        if (z == 0) continue;
        const int dx[5] = {0, -1, 1, 0, 0};
        const int dy[5] = {0, 0, 0, -1, 1};
        for (int k = 0; k < 5; k++) {
            int32_t px = x + dx[k], py = y + dy[k];
            if (px < 0 || px >= nx || py < 0 || py >= ny) continue;
            if (idx) idx[e] = px + nx * (py + ny * (z - 1));
            e++;
        }
    }
    if (ptr) ptr[B] = (int32_t)e;
    return e;
}

/* Ore/waste per (block, scenario) and the block's undiscounted cash flow.
 * Ore <=> processing value beats waste value:
 *   m*(g*p*rec - pc - mc) > -m*mc  <=>  (g*p)*rec > pc   (m > 0 cancels),
 * evaluated as ((g*price)*recovery) > proc_cost with a strict '>'.
 *   value = ore ? m*((g*p)*rec - pc) - m*mc : -m*mc.                       */
void or_classify(const or_model *M, uint8_t *ore, double *value) {
    int64_t BS = (int64_t)M->B * M->S;
    for (int64_t i = 0; i < BS; i++) {
        int64_t b = i / M->S;
        double m = (double)M->mass[b];
        double g = M->grade[i];
        double rev = (g * M->price) * M->recovery;
        int o = rev > M->proc_cost;
        if (ore) ore[i] = (uint8_t)o;
        if (value) value[i] = o ? (m * (rev - M->proc_cost) - m * M->mining_cost) : (-m * M->mining_cost);
    }
}

static double disc(const or_model *M, int t) {
    if (t >= M->T) return 0.0;
    return pow(1.0 + M->discount_rate, -(double)t);
}

/* Mill deviation penalty of one period: a*max(0, Q-O) + e*max(0, O-Q). */
static double penalty(const or_model *M, int t, int64_t ore_t) {
    int64_t q = (int64_t)M->target[t];
    double short_t = ore_t < q ? (double)(q - ore_t) : 0.0;
    double excess_t = ore_t > q ? (double)(ore_t - q) : 0.0;
    return M->shortfall_pen * short_t + M->excess_pen * excess_t;
}

/* Cash flow of block b in scenario s when mined in period t (0 when t = T,
 * unmined).  Without weights it is value[b,s].  With the uncertainty weights
 * of Section 5.6 (Eq. 12: ENPV_{b,s,t} = sigma(s,t) (Revenue - ProcessingCost))
 * the processing margin m((g*p)*rec - pc) of an ore block is scaled by
 * sigma(s,t); the mining cost m*mc (the scenario-independent c_bt of Eq. 14)
 * and the mill penalties are not. */
static double block_cash(const or_model *M, const uint8_t *ore, const double *value, int32_t b, int s, int t) {
    if (t >= M->T) return 0.0;
    int64_t i = (int64_t)b * M->S + s;
    if (!M->sigma) return value[i];
    double m = (double)M->mass[b];
    double margin = ore[i] ? m * ((M->grade[i] * M->price) * M->recovery - M->proc_cost) : 0.0;
    return M->sigma[(int64_t)t * M->S + s] * margin - m * M->mining_cost;
}

/* minedT[t] and oreT[t*S+s] for t < T (integer tonnes, exact). */
void or_tonnage(const or_model *M, const uint8_t *ore, const uint8_t *x, int64_t *minedT, int64_t *oreT) {
    int S = M->S, T = M->T;
    memset(minedT, 0, sizeof(int64_t) * T);
    memset(oreT, 0, sizeof(int64_t) * (size_t)T * S);
    for (int32_t b = 0; b < M->B; b++) {
        int t = x[b];
        if (t >= T) continue;
        minedT[t] += M->mass[b];
        for (int s = 0; s < S; s++)
            if (ore[(int64_t)b * S + s]) oreT[(int64_t)t * S + s] += M->mass[b];
    }
}

/* NPV_s(x) = sum_t d_t * ( sum_{b: x_b = t} cash(b,s,t) - pen_t(oreT[t,s]) ),
 * cash = value[b,s] or its weighted form (block_cash). */
void or_npv(const or_model *M, const uint8_t *ore, const double *value, const uint8_t *x, double *npv) {
    int S = M->S, T = M->T;
    double *cash = (double *)calloc((size_t)T * S, sizeof(double));
    int64_t *oreT = (int64_t *)calloc((size_t)T * S, sizeof(int64_t));
    for (int32_t b = 0; b < M->B; b++) {
        int t = x[b];
        if (t >= T) continue;
        for (int s = 0; s < S; s++) {
            cash[(int64_t)t * S + s] += block_cash(M, ore, value, b, s, t);
            if (ore[(int64_t)b * S + s]) oreT[(int64_t)t * S + s] += M->mass[b];
        }
    }
    for (int s = 0; s < S; s++) {
        double acc = 0.0;
        for (int t = 0; t < T; t++)
            acc += disc(M, t) * (cash[(int64_t)t * S + s] - penalty(M, t, oreT[(int64_t)t * S + s]));
        npv[s] = acc;
    }
    free(cash);
    free(oreT);
}

/* Full feasibility of a schedule: Eq. 15 on every arc, Eq. 16 in every period. */
int or_feasible(const or_model *M, const uint8_t *x) {
    for (int32_t b = 0; b < M->B; b++)
        for (int32_t k = M->pred_ptr[b]; k < M->pred_ptr[b + 1]; k++)
            if (x[M->pred_idx[k]] > x[b]) return 0;
    int64_t *mined = (int64_t *)calloc(M->T, sizeof(int64_t));
    for (int32_t b = 0; b < M->B; b++)
        if (x[b] < M->T) mined[x[b]] += M->mass[b];
    int ok = 1;
    for (int t = 0; t < M->T; t++)
        if ((uint64_t)mined[t] > M->cap[t]) ok = 0;
    free(mined);
    return ok;
}

/* ------------------------------------------------------------- moves */

/* Decode (b1, arg).  Returns 0 for a bad move.  On success fills the moved
 * blocks and their new periods (n_moved = 1 for a shift, 2 for a swap). */
static int decode(const or_model *M, const uint8_t *x, int32_t b1, int32_t arg,
                  int32_t *blk, int *newp, int *n_moved) {
    if (b1 < 0 || b1 >= M->B) return 0;
    if (arg >= 0) {
        if (arg >= M->B) return 0;
        blk[0] = b1; newp[0] = x[arg];
        blk[1] = arg; newp[1] = x[b1];
        *n_moved = 2;
    } else {
        int64_t t = -(int64_t)arg - 1;
        if (t > M->T) return 0;
        blk[0] = b1; newp[0] = (int)t;
        *n_moved = 1;
    }
    return 1;
}

/* Local feasibility flag of a move, brute force: every arc with an end in a
 * moved block holds in x', and every period a moved block leaves or enters
 * is within capacity in x'.  xp is x' (already applied). */
static int brute_flag(const or_model *M, const uint8_t *x, const uint8_t *xp,
                      const int32_t *blk, int n_moved) {
    for (int32_t j = 0; j < M->B; j++) {
        for (int32_t k = M->pred_ptr[j]; k < M->pred_ptr[j + 1]; k++) {
            int32_t p = M->pred_idx[k];
            int touches = 0;
            for (int i = 0; i < n_moved; i++)
                if (blk[i] == p || blk[i] == j) touches = 1;
            if (touches && xp[p] > xp[j]) return 0;
        }
    }
    for (int i = 0; i < n_moved; i++) {
        int periods[2] = {x[blk[i]], xp[blk[i]]};
        for (int q = 0; q < 2; q++) {
            int t = periods[q];
            if (t >= M->T) continue;
            int64_t mined = 0;
            for (int32_t b = 0; b < M->B; b++)
                if (xp[b] == t) mined += M->mass[b];
            if ((uint64_t)mined > M->cap[t]) return 0;
        }
    }
    return 1;
}

static void reduce_scores(const or_model *M, const double *d, double *mean, double *std, double *score) {
    int S = M->S;
    double acc = 0.0;
    for (int s = 0; s < S; s++) acc += d[s];
    double mu = acc / S;
    double v = 0.0;
    for (int s = 0; s < S; s++) v += (d[s] - mu) * (d[s] - mu);
    double sd = sqrt(v / S);
    *mean = mu;
    *std = sd;
    *score = mu - M->lambda * sd;
}

static void bad_move_out(const or_model *M, int64_t i, double *delta, double *mean, double *std,
                         double *score, uint8_t *flag) {
    if (delta) memset(delta + i * M->S, 0, sizeof(double) * M->S);
    if (mean) mean[i] = 0.0;
    if (std) std[i] = 0.0;
    if (score) score[i] = -INFINITY;
    if (flag) flag[i] = 0;
}

/* Brute force: Delta_s = NPV_s(x') - NPV_s(x), recomputed in full per move. */
void or_eval_bruteforce(const or_model *M, const uint8_t *ore, const double *value, const uint8_t *x,
                        const int32_t *moves, int64_t n, double *delta, double *mean, double *std,
                        double *score, uint8_t *flag) {
    int S = M->S;
    double *npv0 = (double *)malloc(sizeof(double) * S);
    or_npv(M, ore, value, x, npv0);
#pragma omp parallel
    {
        uint8_t *xp = (uint8_t *)malloc(M->B);
        double *npv1 = (double *)malloc(sizeof(double) * S);
        double *dl = (double *)malloc(sizeof(double) * S);
#pragma omp for schedule(dynamic, 4)
        for (int64_t i = 0; i < n; i++) {
            int32_t blk[2];
            int newp[2], nm = 0;
            if (!decode(M, x, moves[2 * i], moves[2 * i + 1], blk, newp, &nm)) {
                bad_move_out(M, i, delta, mean, std, score, flag);
                continue;
            }
            memcpy(xp, x, M->B);
            for (int k = 0; k < nm; k++) xp[blk[k]] = (uint8_t)newp[k];
            or_npv(M, ore, value, xp, npv1);
            for (int s = 0; s < S; s++) dl[s] = npv1[s] - npv0[s];
            double mu, sd, sc;
            reduce_scores(M, dl, &mu, &sd, &sc);
            if (delta) memcpy(delta + i * S, dl, sizeof(double) * S);
            if (mean) mean[i] = mu;
            if (std) std[i] = sd;
            if (score) score[i] = sc;
            if (flag) flag[i] = (uint8_t)brute_flag(M, x, xp, blk, nm);
        }
        free(xp);
        free(npv1);
        free(dl);
    }
    free(npv0);
}

/* ------------------------------------------------------- incremental */

/* Second, independent evaluator: O(S) per move from the per-period integer
 * tonnages.  For each moved block c going from period f to period u:
 *   value change   v[c,s] * (d_u - d_f)
 *                  (weighted: cash(c,s,u) d_u - cash(c,s,f) d_f, see block_cash)
 *   ore change     -m_c*ore[c,s] in period f, +m_c*ore[c,s] in period u
 * then for each affected period p < T:
 *   NPV change  -d_p * ( pen_p(O[p,s] + dO[p,s]) - pen_p(O[p,s]) ).
 * floor_s (optional) receives, per scenario, the sum of the magnitudes of the
 * individual terms above; floor (optional) is its mean over scenarios.  These
 * set the scale of an acceptable rounding error near cancellation. */
void or_eval_incremental(const or_model *M, const uint8_t *ore, const double *value, const uint8_t *x,
                         const int32_t *moves, int64_t n, double *delta, double *mean, double *std,
                         double *score, uint8_t *flag, double *floor, double *floor_s) {
    int S = M->S, T = M->T;
    int32_t B = M->B;
    int64_t *minedT = (int64_t *)malloc(sizeof(int64_t) * T);
    int64_t *oreT = (int64_t *)malloc(sizeof(int64_t) * (size_t)T * S);
    or_tonnage(M, ore, x, minedT, oreT);
    double *d = (double *)malloc(sizeof(double) * (T + 1));
    for (int t = 0; t <= T; t++) d[t] = disc(M, t);
    /* successor CSR from the predecessor CSR */
    int64_t E = M->pred_ptr[B];
    int32_t *sptr = (int32_t *)calloc((size_t)B + 1, sizeof(int32_t));
    int32_t *sidx = (int32_t *)malloc(sizeof(int32_t) * (E > 0 ? E : 1));
    for (int64_t k = 0; k < E; k++) sptr[M->pred_idx[k] + 1]++;
    for (int32_t b = 0; b < B; b++) sptr[b + 1] += sptr[b];
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (B > 0 ? B : 1));
    memcpy(fill, sptr, sizeof(int32_t) * B);
    for (int32_t b = 0; b < B; b++)
        for (int32_t k = M->pred_ptr[b]; k < M->pred_ptr[b + 1]; k++) sidx[fill[M->pred_idx[k]]++] = b;
    free(fill);

#pragma omp parallel
    {
        double *dl = (double *)malloc(sizeof(double) * S);
        double *fl = (double *)malloc(sizeof(double) * S);
#pragma omp for schedule(static)
        for (int64_t i = 0; i < n; i++) {
            int32_t blk[2] = {0, 0};
            int newp[2] = {0, 0}, nm = 0;
            if (!decode(M, x, moves[2 * i], moves[2 * i + 1], blk, newp, &nm)) {
                bad_move_out(M, i, delta, mean, std, score, flag);
                if (floor) floor[i] = 0.0;
                if (floor_s) memset(floor_s + i * S, 0, sizeof(double) * S);
                continue;
            }
            int oldp[2];
            for (int k = 0; k < nm; k++) oldp[k] = x[blk[k]];
            /* a swap of a block with itself changes nothing */
            if (nm == 2 && blk[0] == blk[1]) nm = 1, newp[0] = oldp[0];
#define XP(b) ((nm >= 1 && (b) == blk[0]) ? newp[0] : ((nm == 2 && (b) == blk[1]) ? newp[1] : x[b]))
            /* precedence on arcs incident to moved blocks */
            int ok = 1;
            for (int k = 0; k < nm && ok; k++) {
                int32_t c = blk[k];
                int pc = XP(c);
                for (int32_t j = M->pred_ptr[c]; j < M->pred_ptr[c + 1]; j++)
                    if (XP(M->pred_idx[j]) > pc) ok = 0;
                for (int32_t j = sptr[c]; j < sptr[c + 1]; j++)
                    if (pc > XP(sidx[j])) ok = 0;
            }
            /* capacity in every period a moved block leaves or enters */
            int per[4], np = 0;
            for (int k = 0; k < nm; k++) {
                int cand[2] = {oldp[k], newp[k]};
                for (int q = 0; q < 2; q++) {
                    int t = cand[q], dup = 0;
                    if (t >= T) continue;
                    for (int r = 0; r < np; r++) dup |= per[r] == t;
                    if (!dup) per[np++] = t;
                }
            }
            for (int r = 0; r < np && ok; r++) {
                int t = per[r];
                int64_t mt = minedT[t];
                for (int k = 0; k < nm; k++) {
                    if (oldp[k] == t) mt -= M->mass[blk[k]];
                    if (newp[k] == t) mt += M->mass[blk[k]];
                }
                if ((uint64_t)mt > M->cap[t]) ok = 0;
            }
#undef XP
            for (int s = 0; s < S; s++) {
                double dv = 0.0, fs = 0.0;
                for (int k = 0; k < nm; k++) {
                    if (M->sigma) {
                        double gain = block_cash(M, ore, value, blk[k], s, newp[k]) * d[newp[k]];
                        double loss = block_cash(M, ore, value, blk[k], s, oldp[k]) * d[oldp[k]];
                        dv += gain - loss;
                        fs += fabs(gain) + fabs(loss);
                    } else {
                        double term = value[(int64_t)blk[k] * S + s] * (d[newp[k]] - d[oldp[k]]);
                        dv += term;
                        fs += fabs(term);
                    }
                }
                for (int r = 0; r < np; r++) {
                    int t = per[r];
                    int64_t dO = 0;
                    for (int k = 0; k < nm; k++) {
                        int64_t mo = ore[(int64_t)blk[k] * S + s] ? (int64_t)M->mass[blk[k]] : 0;
                        if (oldp[k] == t) dO -= mo;
                        if (newp[k] == t) dO += mo;
                    }
                    int64_t O = oreT[(int64_t)t * S + s];
                    double dp = d[t] * (penalty(M, t, O + dO) - penalty(M, t, O));
                    dv -= dp;
                    fs += fabs(dp);
                }
                dl[s] = dv;
                fl[s] = fs;
            }
            double mu, sd, sc;
            reduce_scores(M, dl, &mu, &sd, &sc);
            if (delta) memcpy(delta + i * S, dl, sizeof(double) * S);
            if (floor_s) memcpy(floor_s + i * S, fl, sizeof(double) * S);
            if (floor) {
                double a = 0.0;
                for (int s = 0; s < S; s++) a += fl[s];
                floor[i] = a / S;
            }
            if (mean) mean[i] = mu;
            if (std) std[i] = sd;
            if (score) score[i] = sc;
            if (flag) flag[i] = (uint8_t)ok;
        }
        free(dl);
        free(fl);
    }
    free(minedT);
    free(oreT);
    free(d);
    free(sptr);
    free(sidx);
}

/* ----------------------------------------------------------------- top-k */

typedef struct {
    double s;
    int32_t i;
} or_key;

static int key_cmp(const void *a, const void *b) {
    const or_key *x = (const or_key *)a, *y = (const or_key *)b;
    if (x->s > y->s) return -1;
    if (x->s < y->s) return 1;
    return (x->i > y->i) - (x->i < y->i);
}

/* The k feasible moves with the largest scores, ties to the lower index. */
int32_t or_topk(const double *score, const uint8_t *flag, int64_t n, int32_t k, int32_t *idx, double *top) {
    or_key *keys = (or_key *)malloc(sizeof(or_key) * (n > 0 ? n : 1));
    int64_t m = 0;
    for (int64_t i = 0; i < n; i++)
        if (flag[i] && !isnan(score[i])) keys[m].s = score[i], keys[m].i = (int32_t)i, m++;
    qsort(keys, (size_t)m, sizeof(or_key), key_cmp);
    int32_t c = (int32_t)(m < k ? m : k);
    for (int32_t j = 0; j < c; j++) {
        if (idx) idx[j] = keys[j].i;
        if (top) top[j] = keys[j].s;
    }
    free(keys);
    return c;
}

/* ------------------------------------------------------------------ apply */

/* Apply one move to x in place.  Returns 0 when applied, 1 when the move's
 * local feasibility flag is 0 (x unchanged), 2 for a bad move. */
int or_apply(const or_model *M, uint8_t *x, int32_t b1, int32_t arg) {
    int32_t blk[2];
    int newp[2], nm = 0;
    if (!decode(M, x, b1, arg, blk, newp, &nm)) return 2;
    uint8_t *xp = (uint8_t *)malloc(M->B);
    memcpy(xp, x, M->B);
    for (int k = 0; k < nm; k++) xp[blk[k]] = (uint8_t)newp[k];
    int ok = brute_flag(M, x, xp, blk, nm);
    if (ok) memcpy(x, xp, M->B);
    free(xp);
    return ok ? 0 : 1;
}

/* ------------------------------------------------------------ violation */

/* Violation magnitudes of each move, for the epsilon-relaxed fitness of
 * Algorithm 2 (fitness = NPV - penalty * max(0, violation - epsilon)).  The
 * paper leaves violation(S) undefined; the reading used here, both parts
 * exact integers that are zero exactly when the move's flag is 1:
 *   capacity excess: over the distinct periods t < T that a moved block
 *     leaves or enters, the sum of max(0, mined'_t - M_t) (tonnes, Eq. 16);
 *   precedence excess: over the moved blocks b, max(0, L_b - x'_b) +
 *     max(0, x'_b - H_b) (periods, Eq. 15), where L_b is the latest period of
 *     a direct predecessor of b and H_b the earliest period of a direct
 *     successor of b in x' (0 and T when there are none).
 * Brute force: x' is formed and every arc and every block is scanned.  A bad
 * move gets -1 in both outputs. */
void or_violation(const or_model *M, const uint8_t *x, const int32_t *moves, int64_t n, int64_t *cap_ex,
                  int32_t *prec_ex) {
#pragma omp parallel
    {
        uint8_t *xp = (uint8_t *)malloc(M->B);
#pragma omp for schedule(dynamic, 16)
        for (int64_t i = 0; i < n; i++) {
            int32_t blk[2];
            int newp[2], nm = 0;
            if (!decode(M, x, moves[2 * i], moves[2 * i + 1], blk, newp, &nm)) {
                cap_ex[i] = -1;
                prec_ex[i] = -1;
                continue;
            }
            if (nm == 2 && blk[0] == blk[1]) nm = 1; /* a block swapped with itself */
            memcpy(xp, x, M->B);
            for (int k = 0; k < nm; k++) xp[blk[k]] = (uint8_t)newp[k];
            /* capacity over the distinct periods left or entered */
            int per[4], np = 0;
            for (int k = 0; k < nm; k++) {
                int cand[2] = {x[blk[k]], xp[blk[k]]};
                for (int q = 0; q < 2; q++) {
                    int seen = 0;
                    for (int r = 0; r < np; r++)
                        if (per[r] == cand[q]) seen = 1;
                    if (!seen) per[np++] = cand[q];
                }
            }
            int64_t ce = 0;
            for (int r = 0; r < np; r++) {
                int t = per[r];
                if (t >= M->T) continue;
                int64_t mined = 0;
                for (int32_t b = 0; b < M->B; b++)
                    if (xp[b] == t) mined += M->mass[b];
                if ((uint64_t)mined > M->cap[t]) ce += mined - (int64_t)M->cap[t];
            }
            /* precedence: bounds of every moved block in x' from all arcs */
            int32_t pe = 0;
            for (int k = 0; k < nm; k++) {
                int32_t b = blk[k];
                int L = 0, H = M->T;
                for (int32_t c = 0; c < M->B; c++)
                    for (int32_t e = M->pred_ptr[c]; e < M->pred_ptr[c + 1]; e++) {
                        int32_t p = M->pred_idx[e];
                        if (c == b && xp[p] > L) L = xp[p];
                        if (p == b && xp[c] < H) H = xp[c];
                    }
                int t = xp[b];
                pe += (L > t ? L - t : 0) + (t > H ? t - H : 0);
            }
            cap_ex[i] = ce;
            prec_ex[i] = pe;
        }
        free(xp);
    }
}

