/*
 * Per-candidate-move search with the tabular magnetic-mirror-descent update
 * (App. E "Search", steps 1-4; Sec. "Test-Time Search via Update
 * Equivalence"), with the uniform belief sampler in place of the belief
 * network and the uniform random policy in place of the move network.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Readings:
 *  R15 Step 1: S configurations of the opponent's hidden pieces per
 *      position; configuration s is the belief sampler's sample s of the
 *      position's stream (R11).
 *  R16 Step 2: one rollout per (legal move j of the searcher in ascending
 *      action order, configuration s).  Its first ply plays move j; plies
 *      d = 1 .. depth-1 take the rollout policy (R19: uniform, or the magnet
 *      policy under OR_ROLLOUT_MAGNET) with Philox at counter
 *      (stream, j*S + s, d, 5<<24).  depth counts the forced move.
 *  R17 Step 3: a rollout's value is +1, -1, 0 for a win, loss or draw of the
 *      searcher and 0 when it is unfinished after depth plies (there is no
 *      value network); q(j) is the mean over the S rollouts of move j (0
 *      when S = 0).  When the caller gives values by action (a value
 *      network's estimates standing in for the rollouts), q(j) is the given
 *      value of move j as a double and no rollout is run.
 *  R18 Step 4: rho (Tab. notation: the magnet policy picks a piece to move
 *      uniformly, then one of its moves uniformly) gives move j the
 *      probability 1 / (pieces with a legal move * legal moves of move j's
 *      piece).  pi_theta is an input distribution over actions (uniform over
 *      the legal moves when absent).  pi_search(j) is proportional to
 *      exp((q(j) + alpha ln rho(j) + beta ln pi_theta(j)) / (alpha + beta)),
 *      evaluated in double as w(j) = exp(z(j) - max z) over the moves in
 *      ascending order and divided by their ascending sum W.  The move played
 *      is the first j whose ascending running sum of w exceeds u*W, with u the
 *      double (word0 >> 5) * 2^-27 + (word1 >> 6) * 2^-53 of Philox at
 *      counter (stream, 0, 0, 6<<24).  A move with pi_theta(j) = 0 gets
 *      probability 0; if every legal move has pi_theta 0 the position is
 *      rejected.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

static int cmp_int(const void* a, const void* b)
{
    int x = *(const int*)a, y = *(const int*)b;
    return (x > y) - (x < y);
}

/* ply d >= 1 of the rollout with counter word c1: the rollout policy's move (R19) */
static int random_move(const or_game* g, const uint32_t key[2], uint32_t stream, uint32_t c1, uint32_t d)
{
    int mv[400];
    int n = or_legal_moves(g, g->ply & 1, mv);
    if (n == 0) return -1;
    qsort(mv, (size_t)n, sizeof(int), cmp_int);
    uint32_t ctr[4] = { stream, c1, d, 5u << 24 };
    uint32_t w[4];
    or_philox4x32_10(ctr, key, w);
    return or_policy_pick(mv, n, w, g->rules.flags & OR_ROLLOUT_MAGNET);
}

int orx_search(const uint8_t* pos, int P, int S, int depth, uint64_t seed, const uint32_t* stream_ids,
               const float* pi_theta, const float* q_given, double alpha, double beta, int k, int cap, int flags,
               int32_t* n_moves, int16_t* actions, int32_t* tallies, double* q, double* pi, int16_t* chosen,
               uint8_t* status)
{
    or_rules rules;
    rules.battleless_limit = k;
    rules.max_plies = cap;
    rules.flags = flags;
    const uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    or_game* root = (or_game*)malloc(sizeof(or_game));
    or_game* g = (or_game*)malloc(sizeof(or_game));
    for (int p = 0; p < P; ++p) {
        int16_t* act = actions + (size_t)p * OR_SEARCH_MAX_MOVES;
        int32_t* tl = tallies + (size_t)p * OR_SEARCH_MAX_MOVES * 4;
        double* qp = q + (size_t)p * OR_SEARCH_MAX_MOVES;
        double* pp = pi + (size_t)p * OR_SEARCH_MAX_MOVES;
        memset(act, 0xFF, OR_SEARCH_MAX_MOVES * sizeof(int16_t));
        memset(tl, 0, OR_SEARCH_MAX_MOVES * 4 * sizeof(int32_t));
        memset(qp, 0, OR_SEARCH_MAX_MOVES * sizeof(double));
        memset(pp, 0, OR_SEARCH_MAX_MOVES * sizeof(double));
        n_moves[p] = 0;
        chosen[p] = -1;
        status[p] = 0;
        if (or_import(root, pos + (size_t)p * OR_POS_BYTES, &rules, 0)) { status[p] = 1; continue; }
        const uint32_t stream = stream_ids ? stream_ids[p] : (uint32_t)p;
        const int searcher = root->ply & 1, opp = 1 - searcher;
        /* the searcher's legal moves, ascending */
        int mv[400];
        int n = or_legal_moves(root, searcher, mv);
        qsort(mv, (size_t)n, sizeof(int), cmp_int);
        if (n > OR_SEARCH_MAX_MOVES) { free(root); free(g); return -(1 + p); }
        n_moves[p] = n;
        for (int j = 0; j < n; ++j) act[j] = (int16_t)mv[j];
        if (n == 0) continue;
        /* step 1 and 2: configurations and rollouts with a forced first move */
        for (int s = 0; s < S && !q_given; ++s) {
            uint8_t types[40];
            or_belief_sample_one(root, seed, stream, (uint32_t)s, types);
            for (int j = 0; j < n; ++j) {
                memcpy(g, root, sizeof(or_game));
                for (int i = 0; i < 40; ++i) g->type[opp * 40 + i] = types[i];
                int winner = -1;
                or_apply(g, mv[j]);
                int code = or_terminal_after(g, &winner);
                for (int d = 1; !code && d < depth; ++d) {
                    int a = random_move(g, key, stream, (uint32_t)(j * S + s), (uint32_t)d);
                    or_apply(g, a);
                    code = or_terminal_after(g, &winner);
                }
                int slot = !code ? 3 : (winner < 0 ? 2 : (winner == searcher ? 0 : 1));
                tl[4 * j + slot]++;
            }
        }
        /* step 3: mean values */
        for (int j = 0; j < n; ++j) {
            if (q_given) qp[j] = (double)q_given[(size_t)p * 10000 + mv[j]];
            else qp[j] = S > 0 ? (double)(tl[4 * j] - tl[4 * j + 1]) / (double)S : 0.0;
        }
        /* step 4: magnet policy, the update, the sampled move */
        int per_from[OR_NSQ];
        memset(per_from, 0, sizeof(per_from));
        for (int j = 0; j < n; ++j) per_from[mv[j] / 100]++;
        int pieces = 0;
        for (int s = 0; s < OR_NSQ; ++s) pieces += per_from[s] > 0;
        double z[OR_SEARCH_MAX_MOVES];
        double zmax = -INFINITY;
        for (int j = 0; j < n; ++j) {
            const double rho = 1.0 / ((double)pieces * (double)per_from[mv[j] / 100]);
            const double pt = pi_theta ? (double)pi_theta[(size_t)p * 10000 + mv[j]] : 1.0 / (double)n;
            z[j] = pt > 0.0 ? (qp[j] + alpha * log(rho) + beta * log(pt)) / (alpha + beta) : -INFINITY;
            if (z[j] > zmax) zmax = z[j];
        }
        if (zmax == -INFINITY) { status[p] = 2; continue; }
        double W = 0.0;
        for (int j = 0; j < n; ++j) {
            const double w = z[j] == -INFINITY ? 0.0 : exp(z[j] - zmax);
            pp[j] = w;
            W += w;
        }
        uint32_t ctr[4] = { stream, 0u, 0u, 6u << 24 };
        uint32_t r[4];
        or_philox4x32_10(ctr, key, r);
        const double u = ((double)(r[0] >> 5) * 67108864.0 + (double)(r[1] >> 6)) / 9007199254740992.0;
        const double t = u * W;
        double c = 0.0;
        int pick = -1;
        for (int j = 0; j < n; ++j) {
            c += pp[j];
            if (pick < 0 && t < c) pick = j;
        }
        if (pick < 0) pick = n - 1;
        chosen[p] = (int16_t)mv[pick];
        for (int j = 0; j < n; ++j) pp[j] /= W;
    }
    free(root);
    free(g);
    return 0;
}
