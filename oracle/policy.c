/*
 * Rollout policies (App. E "Search"): uniform over the legal moves, or the
 * magnet policy rho (Tab. notation: a piece that has a legal move,
 * uniformly, then one of that piece's legal moves, uniformly).
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Reading R19: both policies take their draws from the one Philox counter
 * of the ply; the uniform policy uses word 0 for the index of the move in
 * ascending action order; the magnet policy uses word 0 for the index of
 * the piece among those with a legal move in ascending order of their
 * squares, and word 1 for the index of the move among that piece's legal
 * moves in ascending action order.
 */
#include "oracle.h"

int or_policy_pick(const int* moves, int n, const uint32_t w[4], int magnet)
{
    if (n <= 0) return -1;
    if (!magnet) return moves[or_uniform(w[0], (uint32_t)n)];
    /* the pieces with a legal move: runs of one from-square in the ascending list */
    int pieces = 0;
    for (int j = 0; j < n; ++j)
        if (j == 0 || moves[j] / 100 != moves[j - 1] / 100) ++pieces;
    const int want = (int)or_uniform(w[0], (uint32_t)pieces);
    int run = -1, start = 0;
    for (int j = 0; j < n; ++j) {
        if (j == 0 || moves[j] / 100 != moves[j - 1] / 100) ++run;
        if (run == want) { start = j; break; }
    }
    int m = 0;
    while (start + m < n && moves[start + m] / 100 == moves[start] / 100) ++m;
    return moves[start + (int)or_uniform(w[1], (uint32_t)m)];
}
