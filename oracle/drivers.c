/*
 * Oracle drivers called from Python through ctypes: the environment loop
 * with auto-reset (App. B.1: ApplyActions, SampleRandomLegalAction, boards
 * reset independently), replay of action logs into positions and planes
 * (App. B.1: states reconstructed on demand), belief samples and rollouts
 * (App. E "Search"), and per-position queries used by the tests.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Readings:
 *  R8  The random policy at ply t of episode e in slot i takes word 0 of
 *      Philox at counter (i, e, t, 2<<24) and plays the floor(r*n/2^32)-th
 *      legal action in ascending order of action = from*100 + to.
 *  R9  A step reports the ply index of the action, the red-player reward of
 *      a game that ended on it (+1 red win, -1 blue win, 0 otherwise), the
 *      ending code, and the mask of the acting player of the state left
 *      behind (the next game's first position after an auto-reset).
 *  R10 Rollout ply d from sample k of stream i draws word 0 of Philox at
 *      counter (i, k, d, 4<<24).  Outcomes are tallied from the view of the
 *      player to move at the root: win, loss, draw, unfinished after D plies.
 */
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

static int sort_int(const void* a, const void* b)
{
    int x = *(const int*)a, y = *(const int*)b;
    return (x > y) - (x < y);
}

static int reward_of(int code, int winner)
{
    if (code == END_FLAG || code == END_NO_MOVES) return winner == 0 ? 1 : -1;
    return 0;
}

static or_rules make_rules(int k, int cap, int flags)
{
    or_rules r;
    r.battleless_limit = k;
    r.max_plies = cap;
    r.flags = flags;
    return r;
}

/* The random policy's move (the rules' OR_ROLLOUT_MAGNET bit selects the
 * magnet policy) from the legal moves in ascending action order. */
static int pick_random(const or_game* g, const uint32_t key[2], uint32_t c0, uint32_t c1, uint32_t c2,
                       uint32_t tag, int* n_out)
{
    int mv[400];
    int n = or_legal_moves(g, g->ply & 1, mv);
    *n_out = n;
    if (n == 0) return -1;
    qsort(mv, (size_t)n, sizeof(int), sort_int);
    uint32_t ctr[4] = { c0, c1, c2, tag << 24 };
    uint32_t w[4];
    or_philox4x32_10(ctr, key, w);
    return or_policy_pick(mv, n, w, g->rules.flags & OR_ROLLOUT_MAGNET);
}

/*
 * Reading R20 (setup pool, Sec. "Data Collection"; left-right orientation
 * randomisation, App. "Learned Setups"): side s of a new game at (slot,
 * episode) takes pool entry number uniform(word 0) of Philox at counter
 * (slot, episode, 0, 7<<24 | s), an entry listing the types on the side's
 * 40 setup squares in ascending square order; with mirroring on, the entry
 * is mirrored left-right (file a <-> j) when word 1 is odd.
 */
static void pool_setup(uint64_t seed, uint32_t slot, uint32_t episode, const uint8_t* pool, int M, int mirror,
                       uint8_t types[OR_NPIECE])
{
    const uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    for (int side = 0; side < 2; ++side) {
        const uint32_t ctr[4] = { slot, episode, 0u, (7u << 24) | (uint32_t)side };
        uint32_t w[4];
        or_philox4x32_10(ctr, key, w);
        const uint8_t* e = pool + ((size_t)side * (size_t)M + or_uniform(w[0], (uint32_t)M)) * 40;
        const int flip = mirror && (w[1] & 1u);
        for (int i = 0; i < 40; ++i) {
            const int row = i / 10, col = i % 10;
            types[40 * side + i] = e[10 * row + (flip ? 9 - col : col)];
        }
    }
}

/*
 * A new game of a slot (App. B.1 reset, App. B.4 reset to a non-initial
 * state): the pinned snapshot if the slot has one (reading R21: its
 * history, two-square and chase state come with it), else the pool's
 * setups, else the Philox setup.  Returns nonzero for a corrupt snapshot.
 */
static int new_game(or_game* g, uint64_t seed, uint32_t slot, uint32_t episode, const or_rules* rules,
                    const uint8_t* pool, int M, int mirror, const uint8_t* pin)
{
    uint8_t types[OR_NPIECE];
    if (pin) return or_import(g, pin, rules, 0);
    if (pool) pool_setup(seed, slot, episode, pool, M, mirror, types);
    else or_setup_types(seed, slot, episode, types);
    or_game_init(g, types, rules, 0);
    return 0;
}

/*
 * Run slots [slot0, slot0+n_slots) for n_steps steps each, starting with
 * episode episode0.  Outputs are [n_steps][n_slots] (mask
 * [n_steps][n_slots][1264]); any may be NULL.  stats[n_slots][8]: games
 * ended by code 1..5, plies played, red wins, blue wins.  pool[2][M][40]
 * (or NULL) gives new games their setups; pins[n_slots][784] with pinned[i]
 * != 0 makes slot i start and restart from its snapshot.
 * Returns 0, -(1 + step*n_slots + slot) for an illegal supplied action, or
 * -(1 + n_steps*n_slots + slot) for a corrupt pinned snapshot.
 */
int orx_env_run(uint64_t seed, int slot0, int n_slots, int n_steps,
                int k, int cap, int flags, int autoreset,
                const int16_t* actions_in,
                int16_t* action_out, int8_t* reward_out, uint8_t* done_out, int16_t* ply_out,
                uint8_t* mask_out, uint32_t* stats, uint8_t* final_pos,
                int episode0, const uint8_t* pool, int pool_m, int mirror, const uint8_t* pins,
                const uint8_t* pinned)
{
    or_rules rules = make_rules(k, cap, flags);
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    or_game* g = (or_game*)malloc(sizeof(or_game));
    int mv[400];
    for (int i = 0; i < n_slots; ++i) {
        uint32_t slot = (uint32_t)(slot0 + i);
        uint32_t episode = (uint32_t)episode0;
        const uint8_t* pin = (pins && pinned && pinned[i]) ? pins + (size_t)i * OR_POS_BYTES : NULL;
        if (new_game(g, seed, slot, episode, &rules, pool, pool_m, mirror, pin)) {
            free(g);
            return -(int)(1 + (size_t)n_steps * (size_t)n_slots + (size_t)i);
        }
        int terminated = 0;
        uint32_t st[8] = { 0 };
        for (int t = 0; t < n_steps; ++t) {
            size_t o = (size_t)t * (size_t)n_slots + (size_t)i;
            int action = -1, code = 0, winner = -1, ply_idx = g->ply;
            if (terminated) {
                code = 0;
            } else {
                code = or_start_check(g, &winner);
                if (!code) {
                    int n;
                    if (actions_in && actions_in[o] >= 0) {
                        action = actions_in[o];
                        if (!or_move_legal(g, g->ply & 1, action)) { free(g); return -(int)(1 + o); }
                    } else {
                        action = pick_random(g, key, slot, episode, (uint32_t)g->ply, 2u, &n);
                    }
                    or_apply(g, action);
                    st[5]++;
                    code = or_terminal_after(g, &winner);
                }
            }
            int rew = reward_of(code, winner);
            if (code) {
                st[code - 1]++;
                if (rew > 0) st[6]++;
                if (rew < 0) st[7]++;
            }
            if (action_out) action_out[o] = (int16_t)action;
            if (reward_out) reward_out[o] = (int8_t)rew;
            if (done_out) done_out[o] = (uint8_t)code;
            if (ply_out) ply_out[o] = (int16_t)ply_idx;
            if (code) {
                if (autoreset) {
                    episode++;
                    new_game(g, seed, slot, episode, &rules, pool, pool_m, mirror, pin);
                } else {
                    terminated = 1;
                }
            }
            if (mask_out) {
                uint8_t* m = mask_out + o * OR_MASK_BYTES;
                if (terminated) memset(m, 0, OR_MASK_BYTES);
                else {
                    int n = or_legal_moves(g, g->ply & 1, mv);
                    or_mask_from_moves(mv, n, m);
                }
            }
        }
        if (stats) memcpy(stats + 8 * (size_t)i, st, sizeof(st));
        if (final_pos) or_export(g, final_pos + (size_t)i * OR_POS_BYTES);
    }
    free(g);
    return 0;
}

/* Play the first episode of each slot to its end; record setups and actions. */
int orx_play_games(uint64_t seed, int n_games, int k, int cap, int flags,
                   uint8_t* setups /*[n][80]*/, int16_t* actions /*[n][cap]*/,
                   int32_t* lengths, uint8_t* endings, int8_t* rewards)
{
    or_rules rules = make_rules(k, cap, flags);
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    or_game* g = (or_game*)malloc(sizeof(or_game));
    for (int i = 0; i < n_games; ++i) {
        or_setup_types(seed, (uint32_t)i, 0, setups + 80 * (size_t)i);
        or_game_init(g, setups + 80 * (size_t)i, &rules, 0);
        int16_t* log = actions + (size_t)cap * (size_t)i;
        for (int t = 0; t < cap; ++t) log[t] = -1;
        int winner = -1;
        int code = or_start_check(g, &winner);
        while (!code) {
            int n;
            int a = pick_random(g, key, (uint32_t)i, 0u, (uint32_t)g->ply, 2u, &n);
            log[g->ply] = (int16_t)a;
            or_apply(g, a);
            code = or_terminal_after(g, &winner);
        }
        lengths[i] = g->ply;
        endings[i] = (uint8_t)code;
        rewards[i] = (int8_t)reward_of(code, winner);
    }
    free(g);
    return 0;
}

/* Replay one log prefix with full legality checks.  Returns 0 or -1. */
static int replay(or_game* g, const uint8_t* setup, const int16_t* log, int ply, const or_rules* rules,
                  int track)
{
    or_game_init(g, setup, rules, track);
    for (int t = 0; t < ply; ++t) {
        int w;
        if (or_start_check(g, &w)) return -1;
        if (!or_move_legal(g, g->ply & 1, log[t])) return -1;
        or_apply(g, log[t]);
        if (t + 1 < ply && or_terminal_after(g, &w)) return -1;
    }
    return 0;
}

int orx_replay_positions(const uint8_t* setups, const int16_t* actions, int L,
                         const int32_t* game, const int16_t* ply, int B,
                         int k, int cap, int flags, uint8_t* out_pos)
{
    or_rules rules = make_rules(k, cap, flags);
    or_game* g = (or_game*)malloc(sizeof(or_game));
    for (int b = 0; b < B; ++b) {
        if (replay(g, setups + 80 * (size_t)game[b], actions + (size_t)L * (size_t)game[b], ply[b], &rules, 0)) {
            free(g);
            return -(1 + b);
        }
        or_export(g, out_pos + (size_t)b * OR_POS_BYTES);
    }
    free(g);
    return 0;
}

int orx_obs_encode(const uint8_t* setups, const int16_t* actions, int L,
                   const int32_t* game, const int16_t* ply, const int8_t* player, int B,
                   int k, int cap, int flags,
                   uint8_t* planes, uint16_t* planes_bf16, uint8_t* mask)
{
    or_rules rules = make_rules(k, cap, flags);
    or_game* g = (or_game*)malloc(sizeof(or_game));
    uint8_t* u8 = (uint8_t*)malloc(OR_NCHAN * 100);
    uint16_t* bf = (uint16_t*)malloc(OR_NCHAN * 100 * 2);
    int mv[400];
    for (int b = 0; b < B; ++b) {
        if (replay(g, setups + 80 * (size_t)game[b], actions + (size_t)L * (size_t)game[b], ply[b], &rules, 1)) {
            free(g); free(u8); free(bf);
            return -(1 + b);
        }
        int pl = (player && player[b] >= 0) ? player[b] : (g->ply & 1);
        or_encode_planes(g, pl, u8, bf);
        if (planes) memcpy(planes + (size_t)b * OR_NCHAN * 100, u8, OR_NCHAN * 100);
        if (planes_bf16) memcpy(planes_bf16 + (size_t)b * OR_NCHAN * 100, bf, OR_NCHAN * 100 * 2);
        if (mask) {
            int n = or_legal_moves(g, g->ply & 1, mv);
            or_mask_from_moves(mv, n, mask + (size_t)b * OR_MASK_BYTES);
        }
    }
    free(g); free(u8); free(bf);
    return 0;
}

int orx_belief_sample(const uint8_t* pos, int P, int K, uint64_t seed, const uint32_t* stream_ids,
                      uint8_t* types_out)
{
    or_rules rules = make_rules(100, 1000, 0);
    or_game* g = (or_game*)malloc(sizeof(or_game));
    for (int p = 0; p < P; ++p) {
        if (or_import(g, pos + (size_t)p * OR_POS_BYTES, &rules, 0)) { free(g); return -(1 + p); }
        uint32_t stream = stream_ids ? stream_ids[p] : (uint32_t)p;
        for (int k = 0; k < K; ++k)
            or_belief_sample_one(g, seed, stream, (uint32_t)k, types_out + ((size_t)p * K + k) * 40);
    }
    free(g);
    return 0;
}

int orx_rollout(const uint8_t* pos, int P, int K, int depth, uint64_t seed, const uint32_t* stream_ids,
                const uint8_t* types_in, int k, int cap, int flags, int32_t* tallies, int8_t* outcome_out)
{
    or_rules rules = make_rules(k, cap, flags);
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    or_game* root = (or_game*)malloc(sizeof(or_game));
    or_game* g = (or_game*)malloc(sizeof(or_game));
    for (int p = 0; p < P; ++p) {
        if (or_import(root, pos + (size_t)p * OR_POS_BYTES, &rules, 0)) { free(root); free(g); return -(1 + p); }
        uint32_t stream = stream_ids ? stream_ids[p] : (uint32_t)p;
        int searcher = root->ply & 1, opp = 1 - searcher;
        int32_t tl[4] = { 0, 0, 0, 0 };
        for (int s = 0; s < K; ++s) {
            uint8_t types[40];
            if (types_in) memcpy(types, types_in + ((size_t)p * K + s) * 40, 40);
            else or_belief_sample_one(root, seed, stream, (uint32_t)s, types);
            memcpy(g, root, sizeof(or_game));
            for (int i = 0; i < 40; ++i) g->type[opp * 40 + i] = types[i];
            int winner = -1;
            int code = or_start_check(g, &winner);
            for (int d = 0; !code && d < depth; ++d) {
                int n;
                int a = pick_random(g, key, stream, (uint32_t)s, (uint32_t)d, 4u, &n);
                or_apply(g, a);
                code = or_terminal_after(g, &winner);
            }
            int slot = !code ? 3 : (winner < 0 ? 2 : (winner == searcher ? 0 : 1));
            tl[slot]++;
            if (outcome_out) outcome_out[(size_t)p * K + s] = (int8_t)slot;
        }
        memcpy(tallies + 4 * (size_t)p, tl, sizeof(tl));
    }
    free(root); free(g);
    return 0;
}

/* ---- single-position queries for hand-built test positions ---- */

int orx_legal_moves(const uint8_t* pos, int k, int cap, int flags, int physical, int* moves)
{
    or_rules rules = make_rules(k, cap, flags);
    or_game* g = (or_game*)malloc(sizeof(or_game));
    int n;
    if (or_import(g, pos, &rules, 0)) { free(g); return -1; }
    n = physical ? or_physical_moves(g, g->ply & 1, moves) : or_legal_moves(g, g->ply & 1, moves);
    qsort(moves, (size_t)n, sizeof(int), sort_int);
    free(g);
    return n;
}

/* The rollout policy's move in a position for the words (w0, w1, 0, 0);
 * -1 without a legal move, -2 for an invalid snapshot. */
int orx_policy_pick(const uint8_t* pos, int k, int cap, int flags, uint32_t w0, uint32_t w1)
{
    or_rules rules = make_rules(k, cap, flags);
    or_game* g = (or_game*)malloc(sizeof(or_game));
    int mv[400];
    if (or_import(g, pos, &rules, 0)) { free(g); return -2; }
    const int n = or_legal_moves(g, g->ply & 1, mv);
    qsort(mv, (size_t)n, sizeof(int), sort_int);
    const uint32_t w[4] = { w0, w1, 0u, 0u };
    const int a = or_policy_pick(mv, n, w, flags & OR_ROLLOUT_MAGNET);
    free(g);
    return a;
}

int orx_brute_moves(const uint8_t* pos, int* moves)
{
    or_rules rules = make_rules(100, 1000, 0);
    or_game* g = (or_game*)malloc(sizeof(or_game));
    if (or_import(g, pos, &rules, 0)) { free(g); return -1; }
    int n = or_brute_moves(g, g->ply & 1, moves);
    qsort(moves, (size_t)n, sizeof(int), sort_int);
    free(g);
    return n;
}

/* Apply a list of actions to a position; writes the resulting position and
 * the ending code of the last ply (0 none).  Features are tracked from the
 * given position on, starting from zero bits. Returns 0, or -(1+i) when
 * action i is illegal or follows an ended game. */
int orx_apply(const uint8_t* pos, int k, int cap, int flags, const int16_t* actions, int n,
              uint8_t* out_pos, int* ending, int* winner, uint8_t* planes, uint16_t* planes_bf16)
{
    or_rules rules = make_rules(k, cap, flags);
    or_game* g = (or_game*)malloc(sizeof(or_game));
    if (or_import(g, pos, &rules, 1)) { free(g); return -1000; }
    int code = 0, w = -1;
    for (int i = 0; i < n; ++i) {
        if (code || !or_move_legal(g, g->ply & 1, actions[i])) { free(g); return -(1 + i); }
        or_apply(g, actions[i]);
        code = or_terminal_after(g, &w);
    }
    if (out_pos) or_export(g, out_pos);
    if (ending) *ending = code;
    if (winner) *winner = w;
    if (planes || planes_bf16) {
        uint8_t* u8 = (uint8_t*)malloc(OR_NCHAN * 100);
        uint16_t* bf = (uint16_t*)malloc(OR_NCHAN * 100 * 2);
        or_encode_planes(g, g->ply & 1, u8, bf);
        if (planes) memcpy(planes, u8, OR_NCHAN * 100);
        if (planes_bf16) memcpy(planes_bf16, bf, OR_NCHAN * 100 * 2);
        free(u8); free(bf);
    }
    free(g);
    return 0;
}

int orx_start_check(const uint8_t* pos, int k, int cap, int flags, int* winner)
{
    or_rules rules = make_rules(k, cap, flags);
    or_game* g = (or_game*)malloc(sizeof(or_game));
    if (or_import(g, pos, &rules, 0)) { free(g); return -1; }
    int code = or_start_check(g, winner);
    free(g);
    return code;
}

int orx_two_square_applies(const uint8_t* pos, int k, int cap, int flags)
{
    or_rules rules = make_rules(k, cap, flags);
    or_game* g = (or_game*)malloc(sizeof(or_game));
    if (or_import(g, pos, &rules, 0)) { free(g); return -1; }
    int r = or_two_square_applies(g);
    free(g);
    return r;
}

int orx_import_check(const uint8_t* pos)
{
    or_rules rules = make_rules(100, 1000, 0);
    or_game* g = (or_game*)malloc(sizeof(or_game));
    int r = or_import(g, pos, &rules, 0);
    free(g);
    return r;
}

int orx_marginals(const uint8_t* pos, int side, uint32_t* num, uint32_t* den)
{
    or_rules rules = make_rules(100, 1000, 0);
    or_game* g = (or_game*)malloc(sizeof(or_game));
    if (or_import(g, pos, &rules, 0)) { free(g); return -1; }
    or_side_marginals(g, side, num, den);
    free(g);
    return 0;
}

uint64_t orx_perft(const uint8_t* pos, int depth, int use_brute, int k, int cap, int flags)
{
    or_rules rules = make_rules(k, cap, flags);
    or_game* g = (or_game*)malloc(sizeof(or_game));
    if (or_import(g, pos, &rules, 0)) { free(g); return (uint64_t)-1; }
    uint64_t r = or_perft(g, depth, use_brute);
    free(g);
    return r;
}

void orx_setup_types(uint64_t seed, uint32_t slot, uint32_t episode, uint8_t* types)
{
    or_setup_types(seed, slot, episode, types);
}

void orx_initial_position(const uint8_t* types, uint8_t* out_pos)
{
    or_rules rules = make_rules(100, 1000, 0);
    or_game* g = (or_game*)malloc(sizeof(or_game));
    or_game_init(g, types, &rules, 0);
    or_export(g, out_pos);
    free(g);
}

void orx_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int n)
{
    for (int i = 0; i < n; ++i) or_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

int orx_battle(int ta, int td) { return or_battle(ta, td); }
uint16_t orx_bf16_ratio(uint32_t num, uint32_t den) { return or_bf16_ratio(num, den); }
uint8_t orx_u8_ratio(uint32_t num, uint32_t den) { return or_u8_ratio(num, den); }

void orx_ratio_batch(const uint32_t* num, const uint32_t* den, int n, uint16_t* bf16, uint8_t* u8)
{
    for (int i = 0; i < n; ++i) {
        bf16[i] = or_bf16_ratio(num[i], den[i]);
        u8[i] = or_u8_ratio(num[i], den[i]);
    }
}
