/*
 * CPU oracle for CTC forced alignment (Viterbi over the CTC trellis).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or call
 * this file; only the test suite, the smoke check and the CPU baseline leg of
 * the benchmark do. It shares no code, header, table or constant with the CUDA
 * path.
 *
 * What it computes (TorchAudio 2.1 paper, Sec. 4, paragraph "CTC-based forced
 * alignment": frame-level alignment of a CTC emission matrix to a transcript;
 * the CTC trellis itself is the one of Graves et al., cited in Sec. 1):
 *
 *   states s = 0 .. S-1, S = 2L+1, ext[s] = blank for even s, targets[(s-1)/2]
 *   for odd s. A state path is monotone with steps of 0 (stay), 1 (advance) or
 *   2 (skip); a skip is allowed only into an odd state s >= 3 whose label
 *   differs from ext[s-2]. It starts in state 0 or 1 and ends in S-1 or S-2.
 *   The aligned frame labels are ext[s_t]; the alignment maximises the sum of
 *   lp[t][ext[s_t]] over t.
 *
 * The plain dynamic programme below follows that definition directly:
 *   alpha_0(0) = lp[0][blank], alpha_0(1) = lp[0][ext[1]] (if L >= 1),
 *   alpha_0(s) = -inf otherwise;
 *   alpha_t(s) = max(alpha_{t-1}(s), alpha_{t-1}(s-1), alpha_{t-1}(s-2) if skip
 *                allowed) + lp[t][ext[s]].
 * Readings where the paper is silent (they are the contract of this oracle):
 *   - ties inside the max keep the earlier candidate in the order stay,
 *     advance, skip (strict ">" comparisons in that order);
 *   - the final state is S-1 unless alpha_{T-1}(S-2) is strictly greater;
 *   - scores[t] = lp[t][path[t]] and total = alpha_{T-1}(final), which equals
 *     the left-to-right FP32 sum of scores starting from scores[0];
 *   - the input is infeasible when T < L + R, R the number of adjacent equal
 *     targets; a finite problem whose best score is -inf has no path.
 * Rounding: one IEEE round-to-nearest add per cell after an exact max. Build
 * with -O2 -ffp-contract=off and without -ffast-math so the host arithmetic
 * is plain IEEE binary32 / binary64.
 *
 * Memory: the dense form keeps one uint8 backpointer per cell (T*S bytes).
 * When that exceeds max_bp_bytes, the same recursion is run twice: a first
 * pass keeps alpha rows every K frames, a second pass recomputes each segment
 * from its stored row (last segment first) and walks back through it. Both
 * modes produce identical outputs; the second exists only so the oracle can
 * handle hour-long inputs with bounded host memory.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_E_INVAL (-1)
#define OR_E_TARGET (-2)
#define OR_E_INFEASIBLE (-3)
#define OR_E_NOPATH (-6)
#define OR_E_NOMEM (-10)

/* Step A1: validate the problem; writes the adjacent-repeat count R. */
int oracle_validate(const int32_t *targets, int64_t L, int64_t C, int32_t blank,
                    int64_t T, int64_t *repeats_out) {
    int64_t i, R = 0;
    if (T < 1 || C < 2 || L < 0 || blank < 0 || blank >= C) return OR_E_INVAL;
    if (L > 0 && targets == NULL) return OR_E_INVAL;
    for (i = 0; i < L; ++i) {
        if (targets[i] < 0 || targets[i] >= C || targets[i] == blank) return OR_E_TARGET;
        if (i > 0 && targets[i] == targets[i - 1]) ++R;
    }
    if (repeats_out) *repeats_out = R;
    if (T < L + R) return OR_E_INFEASIBLE;
    return OR_OK;
}

static int32_t ext_of(const int32_t *targets, int32_t blank, int64_t s) {
    return (s % 2 == 0) ? blank : targets[(s - 1) / 2];
}

static int skip_allowed(const int32_t *targets, int32_t blank, int64_t s) {
    if (s % 2 == 0 || s < 3) return 0;
    return ext_of(targets, blank, s) != ext_of(targets, blank, s - 2);
}

/* ---------------------------------------------------------------- FP32 -- */

/* One frame of the recursion: cur from prev at frame t; codes to bp (may be NULL). */
static void step_f32(const float *lp_row, const int32_t *targets, int32_t blank, int64_t S,
                     const float *prev, float *cur, uint8_t *bp) {
    int64_t s;
    for (s = 0; s < S; ++s) {
        float best = prev[s];
        uint8_t code = 0;
        if (s >= 1 && prev[s - 1] > best) {
            best = prev[s - 1];
            code = 1;
        }
        if (skip_allowed(targets, blank, s) && prev[s - 2] > best) {
            best = prev[s - 2];
            code = 2;
        }
        cur[s] = best + lp_row[ext_of(targets, blank, s)];
        if (bp) bp[s] = code;
    }
}

static void init_f32(const float *lp_row0, const int32_t *targets, int32_t blank, int64_t S,
                     float *alpha) {
    int64_t s;
    for (s = 0; s < S; ++s) alpha[s] = -INFINITY;
    alpha[0] = lp_row0[blank];
    if (S > 1) alpha[1] = lp_row0[ext_of(targets, blank, 1)];
}

static int64_t final_state_f32(const float *alpha, int64_t S) {
    if (S == 1) return 0;
    return (alpha[S - 2] > alpha[S - 1]) ? S - 2 : S - 1;
}

/*
 * Steps A2-A7 (and A8 when the dense backpointers exceed max_bp_bytes).
 * lp: [T][C] row-major FP32. Outputs (caller-allocated, length T): path (token
 * ids), states (trellis states; may be NULL), scores (lp of the chosen token).
 * total: alpha_{T-1}(final). Returns OR_OK, a validation error, OR_E_NOPATH
 * (outputs still written, total = -inf) or OR_E_NOMEM.
 */
int oracle_viterbi_f32(const float *lp, int64_t T, int64_t C, const int32_t *targets, int64_t L,
                       int32_t blank, int64_t max_bp_bytes, int32_t *path, int32_t *states,
                       float *scores, float *total) {
    int64_t R, S = 2 * L + 1, t, s_cur;
    int rc = oracle_validate(targets, L, C, blank, T, &R);
    float *prev, *cur, *tmp;
    if (rc != OR_OK) return rc;
    prev = (float *)malloc(sizeof(float) * S);
    cur = (float *)malloc(sizeof(float) * S);
    if (!prev || !cur) {
        free(prev);
        free(cur);
        return OR_E_NOMEM;
    }

    if ((double)T * (double)S <= (double)max_bp_bytes) {
        /* Dense backpointers: bp[t*S + s] for t >= 1. */
        uint8_t *bp = (uint8_t *)malloc((size_t)(T * S));
        if (!bp) {
            free(prev);
            free(cur);
            return OR_E_NOMEM;
        }
        init_f32(lp, targets, blank, S, prev);
        for (t = 1; t < T; ++t) {
            step_f32(lp + t * C, targets, blank, S, prev, cur, bp + t * S);
            tmp = prev, prev = cur, cur = tmp;
        }
        s_cur = final_state_f32(prev, S);
        *total = prev[s_cur];
        for (t = T - 1; t >= 0; --t) {
            int32_t tok = ext_of(targets, blank, s_cur);
            if (states) states[t] = (int32_t)s_cur;
            path[t] = tok;
            scores[t] = lp[t * C + tok];
            if (t > 0) s_cur -= bp[t * S + s_cur];
        }
        free(bp);
    } else {
        /* Segment recompute: alpha rows kept at frames 0, K, 2K, ... */
        int64_t K = (int64_t)ceil(sqrt((double)T)), nck, c;
        float *ck;
        uint8_t *seg;
        if (K < 1) K = 1;
        nck = (T - 1) / K + 1;
        ck = (float *)malloc(sizeof(float) * (size_t)(nck * S));
        seg = (uint8_t *)malloc((size_t)(K * S));
        if (!ck || !seg) {
            free(ck);
            free(seg);
            free(prev);
            free(cur);
            return OR_E_NOMEM;
        }
        init_f32(lp, targets, blank, S, prev);
        memcpy(ck, prev, sizeof(float) * S);
        for (t = 1; t < T; ++t) {
            step_f32(lp + t * C, targets, blank, S, prev, cur, NULL);
            tmp = prev, prev = cur, cur = tmp;
            if (t % K == 0) memcpy(ck + (t / K) * S, prev, sizeof(float) * S);
        }
        s_cur = final_state_f32(prev, S);
        *total = prev[s_cur];
        /* Segment c covers frames cK .. e (e = min(cK+K, T-1)); its codes are
           those of frames cK+1 .. e. Walk back from e to cK. */
        for (c = nck - 1; c >= 0; --c) {
            int64_t t0 = c * K, e = t0 + K < T - 1 ? t0 + K : T - 1;
            memcpy(prev, ck + c * S, sizeof(float) * S);
            for (t = t0 + 1; t <= e; ++t) {
                step_f32(lp + t * C, targets, blank, S, prev, cur, seg + (t - t0 - 1) * S);
                tmp = prev, prev = cur, cur = tmp;
            }
            for (t = e; t >= t0; --t) {
                int32_t tok;
                if (t < e || c == nck - 1) {
                    tok = ext_of(targets, blank, s_cur);
                    if (states) states[t] = (int32_t)s_cur;
                    path[t] = tok;
                    scores[t] = lp[t * C + tok];
                }
                if (t > t0) s_cur -= seg[(t - t0 - 1) * S + s_cur];
            }
        }
        free(ck);
        free(seg);
    }
    free(prev);
    free(cur);
    return (*total == -INFINITY) ? OR_E_NOPATH : OR_OK;
}

/*
 * Forward pass only: the best total, no path. Memory O(S). Used where only the
 * score of a huge problem is compared.
 */
int oracle_viterbi_total_f32(const float *lp, int64_t T, int64_t C, const int32_t *targets,
                             int64_t L, int32_t blank, float *total, int32_t *final_state) {
    int64_t R, S = 2 * L + 1, t, f;
    int rc = oracle_validate(targets, L, C, blank, T, &R);
    float *prev, *cur, *tmp;
    if (rc != OR_OK) return rc;
    prev = (float *)malloc(sizeof(float) * S);
    cur = (float *)malloc(sizeof(float) * S);
    if (!prev || !cur) {
        free(prev);
        free(cur);
        return OR_E_NOMEM;
    }
    init_f32(lp, targets, blank, S, prev);
    for (t = 1; t < T; ++t) {
        step_f32(lp + t * C, targets, blank, S, prev, cur, NULL);
        tmp = prev, prev = cur, cur = tmp;
    }
    f = final_state_f32(prev, S);
    *total = prev[f];
    if (final_state) *final_state = (int32_t)f;
    free(prev);
    free(cur);
    return (*total == -INFINITY) ? OR_E_NOPATH : OR_OK;
}

/* ---------------------------------------------------------------- FP64 -- */
/* The same recursion on the FP32 emissions promoted to binary64 (dense only). */
int oracle_viterbi_f64(const float *lp, int64_t T, int64_t C, const int32_t *targets, int64_t L,
                       int32_t blank, int32_t *path, int32_t *states, double *scores,
                       double *total) {
    int64_t R, S = 2 * L + 1, t, s, s_cur;
    int rc = oracle_validate(targets, L, C, blank, T, &R);
    double *prev, *cur, *tmp;
    uint8_t *bp;
    if (rc != OR_OK) return rc;
    prev = (double *)malloc(sizeof(double) * S);
    cur = (double *)malloc(sizeof(double) * S);
    bp = (uint8_t *)malloc((size_t)(T * S));
    if (!prev || !cur || !bp) {
        free(prev);
        free(cur);
        free(bp);
        return OR_E_NOMEM;
    }
    for (s = 0; s < S; ++s) prev[s] = -INFINITY;
    prev[0] = (double)lp[blank];
    if (S > 1) prev[1] = (double)lp[ext_of(targets, blank, 1)];
    for (t = 1; t < T; ++t) {
        const float *row = lp + t * C;
        for (s = 0; s < S; ++s) {
            double best = prev[s];
            uint8_t code = 0;
            if (s >= 1 && prev[s - 1] > best) {
                best = prev[s - 1];
                code = 1;
            }
            if (skip_allowed(targets, blank, s) && prev[s - 2] > best) {
                best = prev[s - 2];
                code = 2;
            }
            cur[s] = best + (double)row[ext_of(targets, blank, s)];
            bp[t * S + s] = code;
        }
        tmp = prev, prev = cur, cur = tmp;
    }
    s_cur = (S == 1) ? 0 : ((prev[S - 2] > prev[S - 1]) ? S - 2 : S - 1);
    *total = prev[s_cur];
    for (t = T - 1; t >= 0; --t) {
        int32_t tok = ext_of(targets, blank, s_cur);
        if (states) states[t] = (int32_t)s_cur;
        path[t] = tok;
        scores[t] = (double)lp[t * C + tok];
        if (t > 0) s_cur -= bp[t * S + s_cur];
    }
    free(prev);
    free(cur);
    free(bp);
    return (*total == -INFINITY) ? OR_E_NOPATH : OR_OK;
}

/*
 * Sum-product variant (the same trellis with log-add in place of max): the
 * log of the total probability of every CTC path that collapses to the
 * transcript, the forward score of the CTC work the paper cites:
 *   beta_0(0) = lp[0][blank], beta_0(1) = lp[0][ext[1]] (if L >= 1), else -inf;
 *   beta_t(s) = log( exp beta_{t-1}(s) + exp beta_{t-1}(s-1)
 *                    + [skip allowed] exp beta_{t-1}(s-2) ) + lp[t][ext[s]];
 *   total = log( exp beta_{T-1}(S-1) + [S > 1] exp beta_{T-1}(S-2) ).
 * In binary64 with the maximum factored out of each log-sum (log sum exp(x) =
 * m + log sum exp(x - m)); a sum of only -inf terms is -inf.
 */
/*
 * Largest |beta_t(s)| over the finite states that can still reach a final
 * state (S-1 or S-2) in the frames left: a path advances at most two states
 * per frame, so s + 2 (T-1-t) >= S-2 (a superset of the states the total
 * depends on). Feeds error bounds only; 0 when no such state is finite.
 */
static double live_abs_max(const double *beta, int64_t S, int64_t T, int64_t t) {
    double m = 0.0;
    int64_t s, lo = S - 2 - 2 * (T - 1 - t);
    if (lo < 0) lo = 0;
    for (s = lo; s < S; ++s)
        if (isfinite(beta[s]) && fabs(beta[s]) > m) m = fabs(beta[s]);
    return m;
}

static double log_add3(double x, double y, double z) {
    double m = x;
    if (y > m) m = y;
    if (z > m) m = z;
    if (m == -INFINITY) return -INFINITY;
    return m + log(exp(x - m) + exp(y - m) + exp(z - m));
}

int oracle_ctc_forward_f64(const float *lp, int64_t T, int64_t C, const int32_t *targets, int64_t L,
                           int32_t blank, double *total, double *amax) {
    int64_t R, S = 2 * L + 1, t, s;
    int rc = oracle_validate(targets, L, C, blank, T, &R);
    double *prev, *cur, *tmp;
    if (rc != OR_OK) return rc;
    prev = (double *)malloc(sizeof(double) * S);
    cur = (double *)malloc(sizeof(double) * S);
    if (!prev || !cur) {
        free(prev);
        free(cur);
        return OR_E_NOMEM;
    }
    for (s = 0; s < S; ++s) prev[s] = -INFINITY;
    prev[0] = (double)lp[blank];
    if (S > 1) prev[1] = (double)lp[ext_of(targets, blank, 1)];
    if (amax) amax[0] = live_abs_max(prev, S, T, 0);
    for (t = 1; t < T; ++t) {
        const float *row = lp + t * C;
        for (s = 0; s < S; ++s) {
            double a1 = (s >= 1) ? prev[s - 1] : -INFINITY;
            double a2 = skip_allowed(targets, blank, s) ? prev[s - 2] : -INFINITY;
            cur[s] = log_add3(prev[s], a1, a2) + (double)row[ext_of(targets, blank, s)];
        }
        tmp = prev, prev = cur, cur = tmp;
        if (amax) amax[t] = live_abs_max(prev, S, T, t);
    }
    *total = log_add3(prev[S - 1], (S > 1) ? prev[S - 2] : -INFINITY, -INFINITY);
    free(prev);
    free(cur);
    return (*total == -INFINITY) ? OR_E_NOPATH : OR_OK;
}
