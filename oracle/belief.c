/*
 * Oracle belief sampler (App. E "Search", first step; Sec. "Test-Time
 * Search"): one assignment of types to the opponent's hidden pieces, drawn
 * uniformly (up to the multiply-shift draw) from the assignments consistent
 * with the public history.  The paper draws these from a trained belief
 * network; without weights the uniform posterior stands in for it.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Constraints (from the public history): revealed and captured pieces have
 * their known type; an unrevealed piece that once moved more than one square
 * is a Scout; an unrevealed piece that moved is neither Bomb nor Flag; the
 * remaining counts of each type are respected.
 *
 * Algorithm (our reading; the paper fixes no sampler):
 *   U = unrevealed unmoved non-Scout-known pieces in ascending square order,
 *   M = unrevealed moved non-Scout-known pieces, counts c_T, b = c_F + c_B,
 *   m = sum of movable c_T.
 *   1. Partial Fisher-Yates over the indices of U: for i = 0..b-1,
 *      j = i + U[0, |U|-i), swap; U[idx[i]] gets Flag for i < c_F, else Bomb.
 *   2. The movable multiset sorted by type code is Fisher-Yates shuffled
 *      (i = m-1..1, j = U[0, i+1)) and laid on M and the unselected U pieces
 *      in ascending square order.
 *   Draw w is word w%4 of Philox at counter (stream, sample, 0, 3<<24 | w/4).
 */
#include <string.h>
#include "oracle.h"

static const int TYPE_COUNT[T_NTYPES] = { 1, 8, 5, 4, 4, 4, 3, 2, 1, 1, 1, 6 };

typedef struct {
    uint32_t key[2];
    uint32_t stream, sample, w;
} draw_stream;

static uint32_t next_word(draw_stream* ds)
{
    uint32_t ctr[4] = { ds->stream, ds->sample, 0u, (3u << 24) | (ds->w >> 2) };
    uint32_t out[4];
    or_philox4x32_10(ctr, ds->key, out);
    uint32_t r = out[ds->w & 3];
    ds->w++;
    return r;
}

void or_belief_sample_one(const or_game* g, uint64_t seed, uint32_t stream, uint32_t sample,
                          uint8_t out[40])
{
    int opp = 1 - (g->ply & 1);
    int c[T_NTYPES];
    for (int t = 0; t < T_NTYPES; ++t) c[t] = TYPE_COUNT[t];
    int slot_u[40], slot_m[40], nU = 0, nM = 0, nS = 0;
    /* pieces in ascending square order: walk the board */
    for (int k = 0; k < 40; ++k) {
        int p = opp * 40 + k;
        if (!g->alive[p] || g->revealed[p]) { out[k] = g->type[p]; c[g->type[p]]--; }
        else if (g->scout_known[p]) { out[k] = T_SCOUT; nS++; }
        else out[k] = 0xFF;
    }
    c[T_SCOUT] -= nS;
    for (int s = 0; s < OR_NSQ; ++s) {
        int p = g->board[s];
        if (p < 0 || p / 40 != opp || out[p - 40 * opp] != 0xFF) continue;
        if (g->moved[p]) slot_m[nM++] = p - 40 * opp;
        else slot_u[nU++] = p - 40 * opp;
    }
    int b = c[T_FLAG] + c[T_BOMB];
    int m = 0;
    for (int t = 0; t <= T_MARSHAL; ++t) m += c[t];

    draw_stream ds = { { (uint32_t)seed, (uint32_t)(seed >> 32) }, stream, sample, 0 };

    /* 1. immovable pieces onto b of the unmoved slots */
    int idx[40], selected[40];
    for (int i = 0; i < nU; ++i) { idx[i] = i; selected[i] = 0; }
    for (int i = 0; i < b && i < nU; ++i) {
        int j = i + (int)or_uniform(next_word(&ds), (uint32_t)(nU - i));
        int tmp = idx[i]; idx[i] = idx[j]; idx[j] = tmp;
        out[slot_u[idx[i]]] = (uint8_t)(i < c[T_FLAG] ? T_FLAG : T_BOMB);
        selected[idx[i]] = 1;
    }

    /* 2. movable multiset over the remaining hidden slots in square order */
    uint8_t arr[40];
    int na = 0;
    for (int t = 0; t <= T_MARSHAL; ++t)
        for (int k = 0; k < c[t]; ++k) arr[na++] = (uint8_t)t;
    for (int i = m - 1; i >= 1; --i) {
        int j = (int)or_uniform(next_word(&ds), (uint32_t)(i + 1));
        uint8_t tmp = arr[i]; arr[i] = arr[j]; arr[j] = tmp;
    }
    int next = 0;
    for (int s = 0; s < OR_NSQ; ++s) {
        int p = g->board[s];
        if (p < 0 || p / 40 != opp) continue;
        int k = p - 40 * opp;
        int is_u = -1;
        for (int i = 0; i < nU; ++i) if (slot_u[i] == k) is_u = i;
        int is_m = 0;
        for (int i = 0; i < nM; ++i) if (slot_m[i] == k) is_m = 1;
        if (is_m || (is_u >= 0 && !selected[is_u])) {
            if (next < na) out[k] = arr[next];
            next++;
        }
    }
}
