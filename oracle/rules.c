/*
 * Oracle game engine: board, pieces, movement, battles, the two-square and
 * continuous-chasing rules, the k-move rule, endings, feature tracking and
 * the position snapshot.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Readings (the paper is silent or loose on these points):
 *  R1  Square s = 10*row + col; row 0 is red's back row; lakes are c5-d6 and
 *      g5-h6, i.e. squares 42,43,52,53,46,47,56,57 (92 occupiable squares,
 *      App. A "Game Summary").
 *  R2  Red pid i starts on square i, blue pid 40+i on square 60+i.
 *  R3  Setup: each side's sorted 40-piece multiset (type code order, counts of
 *      Tab. pieces) is Fisher-Yates shuffled (i = 39..1, j = U[0,i+1) from
 *      draw number 39-i) and laid on the side's squares in ascending order.
 *      Draw d of side p is word d%4 of Philox at counter
 *      (slot, episode, 0, 1<<24 | p<<8 | d/4).
 *  R4  Battle (Tab. pieces): defender Flag -> attacker wins; defender Bomb ->
 *      attacker wins iff Miner; Spy attacking Marshal wins; otherwise the
 *      higher rank wins and equal ranks both die.  Survivors are revealed.
 *  R5  Two-square rule (App. A, App. B.2): a player's next move of the piece
 *      it moved on its last three consecutive turns is illegal when all four
 *      moves lie on one row or one column and some square boundary is crossed
 *      by all four of them (max of the lower ends < min of the upper ends).
 *  R6  Threat = non-battle move ending orthogonally next to an enemy piece.
 *      Evade = non-battle move of a piece that stood next to the square the
 *      opponent's previous (non-battle) move ended on, ending not next to it.
 *      Evade takes precedence.  Chase state: a threat by P continues the chase
 *      when P is already the chaser, else starts one; an evade by the chased
 *      player keeps it; any other ply ends it.  While P chases, a threat whose
 *      resulting position (piece id per square) equals a position reached
 *      after one of P's threats in the chase is illegal, unless it moves the
 *      piece P moved on its previous turn back to that move's from-square
 *      (Tab. chase and the rule below it).
 *  R7  Endings, checked after every ply in this order: flag captured (mover
 *      wins); the next player has no legal move (mover wins, or a draw if the
 *      mover has no physically possible move either); k consecutive
 *      battleless plies (draw); the game-length cap (draw).  A fresh position
 *      whose acting player cannot move ends at once the same way.
 */
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

static int row_of(int s) { return s / 10; }
static int col_of(int s) { return s % 10; }
static int owner_of(int pid) { return pid / 40; }
static int is_movable_type(int t) { return t <= T_MARSHAL; }

int or_is_lake(int s)
{
    return s == 42 || s == 43 || s == 46 || s == 47 ||
           s == 52 || s == 53 || s == 56 || s == 57;
}

static int adjacent(int a, int b)
{
    int dr = row_of(a) - row_of(b), dc = col_of(a) - col_of(b);
    if (dr < 0) dr = -dr;
    if (dc < 0) dc = -dc;
    return dr + dc == 1;
}

/* Orthogonal neighbours that are on the board and not lakes. */
static int neighbours(int s, int out[4])
{
    int n = 0, r = row_of(s), c = col_of(s);
    if (r > 0 && !or_is_lake(s - 10)) out[n++] = s - 10;
    if (r < 9 && !or_is_lake(s + 10)) out[n++] = s + 10;
    if (c > 0 && !or_is_lake(s - 1)) out[n++] = s - 1;
    if (c < 9 && !or_is_lake(s + 1)) out[n++] = s + 1;
    return n;
}

/* Piece counts per type (Tab. pieces), in type code order. */
static const int TYPE_COUNT[T_NTYPES] = { 1, 8, 5, 4, 4, 4, 3, 2, 1, 1, 1, 6 };

int or_battle(int ta, int td)
{
    if (td == T_FLAG) return 1;
    if (td == T_BOMB) return ta == T_MINER ? 1 : 2;
    if (ta == T_SPY && td == T_MARSHAL) return 1;
    if (ta > td) return 1;          /* codes 0-9 are ranks 1-10 in order */
    if (ta < td) return 2;
    return 3;
}

void or_setup_types(uint64_t seed, uint32_t slot, uint32_t episode, uint8_t types[OR_NPIECE])
{
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    for (int side = 0; side < 2; ++side) {
        uint8_t arr[40];
        int n = 0;
        for (int t = 0; t < T_NTYPES; ++t)
            for (int c = 0; c < TYPE_COUNT[t]; ++c)
                arr[n++] = (uint8_t)t;
        for (int i = 39; i >= 1; --i) {
            int d = 39 - i;
            uint32_t ctr[4] = { slot, episode, 0u, (1u << 24) | ((uint32_t)side << 8) | (uint32_t)(d / 4) };
            uint32_t w[4];
            or_philox4x32_10(ctr, key, w);
            uint32_t j = or_uniform(w[d % 4], (uint32_t)(i + 1));
            uint8_t tmp = arr[i]; arr[i] = arr[j]; arr[j] = tmp;
        }
        for (int k = 0; k < 40; ++k) types[side * 40 + k] = arr[k];
    }
}

static void rebuild_board(or_game* g)
{
    for (int s = 0; s < OR_NSQ; ++s) g->board[s] = or_is_lake(s) ? -2 : -1;
    for (int p = 0; p < OR_NPIECE; ++p)
        if (g->alive[p]) g->board[g->sq[p]] = p;
}

void or_game_init(or_game* g, const uint8_t types[OR_NPIECE], const or_rules* rules, int track_features)
{
    memset(g, 0, sizeof(*g));
    for (int p = 0; p < OR_NPIECE; ++p) {
        g->type[p] = types[p];
        g->sq[p] = (uint8_t)(p < 40 ? p : 60 + (p - 40));
        g->alive[p] = 1;
    }
    rebuild_board(g);
    g->ts_pid[0] = g->ts_pid[1] = -1;
    for (int i = 0; i < 4; ++i) g->ts_sq[0][i] = g->ts_sq[1][i] = -1;
    g->chaser = -1;
    for (int i = 0; i < OR_HIST; ++i) g->hist[i] = 0xFFFF;
    g->rules = *rules;
    g->track_features = track_features;
}

/* ---------------------------------------------------------------- moves */

int or_physical_moves(const or_game* g, int player, int* moves)
{
    static const int DR[4] = { 1, -1, 0, 0 };
    static const int DC[4] = { 0, 0, 1, -1 };
    int n = 0;
    for (int p = player * 40; p < player * 40 + 40; ++p) {
        if (!g->alive[p] || !is_movable_type(g->type[p])) continue;
        int s = g->sq[p];
        int maxd = g->type[p] == T_SCOUT ? 9 : 1;
        for (int d = 0; d < 4; ++d) {
            int r = row_of(s), c = col_of(s);
            for (int k = 1; k <= maxd; ++k) {
                r += DR[d]; c += DC[d];
                if (r < 0 || r > 9 || c < 0 || c > 9) break;
                int t = 10 * r + c;
                int occ = g->board[t];
                if (occ == -2) break;                     /* lake */
                if (occ >= 0 && owner_of(occ) == player) break;
                moves[n++] = s * 100 + t;
                if (occ >= 0) break;                      /* enemy: capture ends the slide */
            }
        }
    }
    return n;
}

static int two_square_blocks(const or_game* g, int player, int from, int to)
{
    if (!(g->rules.flags & OR_RULE_TWO_SQUARE)) return 0;
    int pid = g->board[from];
    if (pid < 0 || g->ts_pid[player] != pid || g->ts_len[player] != 4) return 0;
    int sq[5] = { g->ts_sq[player][0], g->ts_sq[player][1], g->ts_sq[player][2],
                  g->ts_sq[player][3], to };
    int same_row = 1, same_col = 1;
    for (int i = 1; i < 5; ++i) {
        if (row_of(sq[i]) != row_of(sq[0])) same_row = 0;
        if (col_of(sq[i]) != col_of(sq[0])) same_col = 0;
    }
    if (!same_row && !same_col) return 0;
    int lo_max = -1, hi_min = 100;
    for (int i = 0; i < 4; ++i) {
        int a = same_row ? col_of(sq[i]) : row_of(sq[i]);
        int b = same_row ? col_of(sq[i + 1]) : row_of(sq[i + 1]);
        int lo = a < b ? a : b, hi = a < b ? b : a;
        if (lo > lo_max) lo_max = lo;
        if (hi < hi_min) hi_min = hi;
    }
    return lo_max < hi_min;
}

enum { CL_BATTLE = 0, CL_QUIET = 1, CL_THREAT = 2, CL_EVADE = 3 };

static int prev_to_square(const or_game* g)
{
    return g->hist[0] == 0xFFFF ? -1 : g->hist[0] % 100;
}

/* Class of a move by `player` from `from` to `to` on the current board (R6). */
static int classify(const or_game* g, int player, int from, int to)
{
    if (g->board[to] >= 0) return CL_BATTLE;
    int a = prev_to_square(g);
    if (a >= 0 && !g->last_battle) {
        int A = g->board[a];
        if (A >= 0 && owner_of(A) != player && adjacent(from, a) && !adjacent(to, a))
            return CL_EVADE;
    }
    int nb[4], nn = neighbours(to, nb);
    for (int i = 0; i < nn; ++i) {
        int q = g->board[nb[i]];
        if (q >= 0 && owner_of(q) != player) return CL_THREAT;
    }
    return CL_QUIET;
}

static void board_bytes(const or_game* g, uint8_t out[OR_NSQ])
{
    for (int s = 0; s < OR_NSQ; ++s) out[s] = g->board[s] >= 0 ? (uint8_t)g->board[s] : 0xFF;
}

static int chase_blocks(const or_game* g, int player, int from, int to)
{
    if (!(g->rules.flags & OR_RULE_CHASE)) return 0;
    if (g->chaser != player || g->n_pi == 0) return 0;
    if (classify(g, player, from, to) != CL_THREAT) return 0;
    /* exception: the piece moved on the chaser's previous turn goes back */
    if (g->hist[1] != 0xFFFF) {
        int pf = g->hist[1] / 100, pt = g->hist[1] % 100;
        if (from == pt && to == pf) return 0;
    }
    uint8_t after[OR_NSQ];
    board_bytes(g, after);
    after[to] = after[from];
    after[from] = 0xFF;
    for (int i = 0; i < g->n_pi; ++i)
        if (memcmp(after, g->pi[i], OR_NSQ) == 0) return 1;
    return 0;
}

int or_legal_moves(const or_game* g, int player, int* moves)
{
    int phys[400];
    int np = or_physical_moves(g, player, phys);
    int n = 0;
    for (int i = 0; i < np; ++i) {
        int from = phys[i] / 100, to = phys[i] % 100;
        if (two_square_blocks(g, player, from, to)) continue;
        if (chase_blocks(g, player, from, to)) continue;
        moves[n++] = phys[i];
    }
    return n;
}

int or_move_legal(const or_game* g, int player, int action)
{
    int mv[400];
    int n = or_legal_moves(g, player, mv);
    for (int i = 0; i < n; ++i) if (mv[i] == action) return 1;
    return 0;
}

void or_mask_from_moves(const int* moves, int n, uint8_t mask[OR_MASK_BYTES])
{
    memset(mask, 0, OR_MASK_BYTES);
    for (int i = 0; i < n; ++i) mask[moves[i] >> 3] |= (uint8_t)(1u << (moves[i] & 7));
}

int or_two_square_applies(const or_game* g)
{
    int player = g->ply & 1;
    int pid = g->ts_pid[player];
    if (pid < 0 || !g->alive[pid]) return 0;
    int phys[400];
    int np = or_physical_moves(g, player, phys);
    for (int i = 0; i < np; ++i)
        if (phys[i] / 100 == g->sq[pid] && two_square_blocks(g, player, phys[i] / 100, phys[i] % 100))
            return 1;
    return 0;
}

/* Independent enumerator: every (piece, direction, distance) triple, with the
 * path checked square by square.  Used only to cross-check move generation. */
int or_brute_moves(const or_game* g, int player, int* moves)
{
    int n = 0;
    for (int s = 0; s < OR_NSQ; ++s) {
        int p = g->board[s];
        if (p < 0 || owner_of(p) != player) continue;
        int t = g->type[p];
        if (t == T_FLAG || t == T_BOMB) continue;
        for (int dir = 0; dir < 4; ++dir) {
            for (int dist = 1; dist <= 9; ++dist) {
                if (dist > 1 && t != T_SCOUT) continue;
                int r = row_of(s), c = col_of(s);
                int ok = 1;
                int dest = -1;
                for (int k = 1; k <= dist; ++k) {
                    int rr = r + (dir == 0 ? k : dir == 1 ? -k : 0);
                    int cc = c + (dir == 2 ? k : dir == 3 ? -k : 0);
                    if (rr < 0 || rr > 9 || cc < 0 || cc > 9) { ok = 0; break; }
                    int q = 10 * rr + cc;
                    if (or_is_lake(q)) { ok = 0; break; }
                    if (k < dist && g->board[q] != -1) { ok = 0; break; }
                    if (k == dist) {
                        if (g->board[q] >= 0 && owner_of(g->board[q]) == player) { ok = 0; break; }
                        dest = q;
                    }
                }
                if (ok) moves[n++] = s * 100 + dest;
            }
        }
    }
    return n;
}

/* ---------------------------------------------------------------- apply */

static void kill_piece(or_game* g, int pid, int square, int cause)
{
    g->alive[pid] = 0;
    g->revealed[pid] = 1;
    g->sq[pid] = (uint8_t)square;
    g->cause[pid] = (uint8_t)cause;
}

/* Feature index of a piece seen by its opponent: 0-9 revealed rank, 10 hidden, -1 none. */
static int idx_rank_or_hidden(const or_game* g, int pid)
{
    if (!g->revealed[pid]) return 10;
    return g->type[pid] <= T_MARSHAL ? g->type[pid] : -1;
}

/* 0-10 revealed Spy..Marshal,Bomb; `hidden_bit` if hidden; -1 for a revealed flag. */
static int idx_type11(const or_game* g, int pid, int hidden_bit)
{
    if (!g->revealed[pid]) return hidden_bit;
    int t = g->type[pid];
    if (t <= T_MARSHAL) return t;
    if (t == T_BOMB) return 10;
    return -1;
}

static void set_bit(uint32_t* w, int bit) { if (bit >= 0) *w |= 1u << bit; }

static void features_before_move(or_game* g, int player, int action)
{
    int from = action / 100, to = action % 100;
    int X = g->board[from];
    int battle = g->board[to] >= 0;
    int nb[4], nn;

    /* active adjacency: adjacent attacks that were legal but not chosen */
    for (int p = player * 40; p < player * 40 + 40; ++p) {
        if (!g->alive[p] || !is_movable_type(g->type[p])) continue;
        int s = g->sq[p];
        nn = neighbours(s, nb);
        for (int i = 0; i < nn; ++i) {
            int Z = g->board[nb[i]];
            if (Z < 0 || owner_of(Z) == player) continue;
            if (s * 100 + nb[i] == action) continue;
            if (two_square_blocks(g, player, s, nb[i])) continue;
            set_bit(&g->f_active[p], idx_rank_or_hidden(g, Z));
        }
    }

    int a = prev_to_square(g);
    if (a < 0 || g->last_battle || battle) return;
    int A = g->board[a];
    if (A < 0 || owner_of(A) == player) return;

    /* evasion of the previous ply's threat */
    if (adjacent(from, a) && !adjacent(to, a))
        set_bit(&g->f_evade[X], idx_rank_or_hidden(g, A));

    /* protection: the previous ply threatened something of ours */
    int threatened = 0;
    nn = neighbours(a, nb);
    for (int i = 0; i < nn; ++i) {
        int q = g->board[nb[i]];
        if (q >= 0 && owner_of(q) == player) threatened = 1;
    }
    if (!threatened) return;
    for (int i = 0; i < nn; ++i) {
        int s = nb[i];
        int B = g->board[s];
        if (B >= 0 && (owner_of(B) != player || B == X)) continue;
        if (!(adjacent(to, s) && !adjacent(from, s))) continue;
        if (B < 0) set_bit(&g->f_prot[X], 11);
        else set_bit(&g->f_prot[X], idx_type11(g, B, 12));
        set_bit(&g->f_pagainst[X], idx_type11(g, A, 11));
        if (B >= 0) {
            set_bit(&g->f_pby[B], idx_type11(g, X, 11));
            set_bit(&g->f_pbyagainst[B], idx_type11(g, A, 11));
        }
    }
}

void or_apply(or_game* g, int action)
{
    int P = g->ply & 1;
    int from = action / 100, to = action % 100;
    int X = g->board[from];
    int cls = classify(g, P, from, to);

    if (g->track_features) features_before_move(g, P, action);

    int dist = row_of(from) == row_of(to) ? col_of(to) - col_of(from) : row_of(to) - row_of(from);
    if (dist < 0) dist = -dist;
    if (dist > 1) g->scout_known[X] = 1;
    g->moved[X] = 1;

    int battle = g->board[to] >= 0;
    int D = -1, d_died = 0;
    if (!battle) {
        g->board[from] = -1;
        g->board[to] = X;
        g->sq[X] = (uint8_t)to;
    } else {
        D = g->board[to];
        int d_was_revealed = g->revealed[D];
        int out = or_battle(g->type[X], g->type[D]);
        g->revealed[X] = 1;
        g->revealed[D] = 1;
        g->board[from] = -1;
        if (out == 1) {
            kill_piece(g, D, to, d_was_revealed ? 4 : 6);
            d_died = 1;
            g->board[to] = X;
            g->sq[X] = (uint8_t)to;
        } else if (out == 2) {
            kill_piece(g, X, to, d_was_revealed ? 1 : 3);
        } else {
            kill_piece(g, X, to, d_was_revealed ? 2 : 3);
            kill_piece(g, D, to, d_was_revealed ? 5 : 6);
            d_died = 1;
            g->board[to] = -1;
        }
    }
    g->battleless = battle ? 0 : g->battleless + 1;
    g->last_battle = battle;
    g->ply += 1;

    /* two-square state (R5) */
    if (!g->alive[X]) {
        g->ts_pid[P] = -1; g->ts_len[P] = 0;
        for (int i = 0; i < 4; ++i) g->ts_sq[P][i] = -1;
    } else if (g->ts_pid[P] == X && g->ts_len[P] >= 2) {
        if (g->ts_len[P] == 4) {
            for (int i = 0; i < 3; ++i) g->ts_sq[P][i] = g->ts_sq[P][i + 1];
            g->ts_sq[P][3] = to;
        } else {
            g->ts_sq[P][g->ts_len[P]++] = to;
        }
    } else {
        g->ts_pid[P] = X; g->ts_len[P] = 2;
        g->ts_sq[P][0] = from; g->ts_sq[P][1] = to; g->ts_sq[P][2] = g->ts_sq[P][3] = -1;
    }
    if (d_died && g->ts_pid[1 - P] == D) {
        g->ts_pid[1 - P] = -1; g->ts_len[1 - P] = 0;
        for (int i = 0; i < 4; ++i) g->ts_sq[1 - P][i] = -1;
    }

    /* chase state (R6) */
    if (cls == CL_THREAT) {
        if (g->chaser != P) { g->chaser = P; g->n_pi = 0; g->chase_plies = 0; }
        if (g->n_pi < OR_MAX_PI) board_bytes(g, g->pi[g->n_pi++]);
        g->chase_plies += 1;
    } else if (cls == CL_EVADE && g->chaser == 1 - P) {
        g->chase_plies += 1;
    } else {
        g->chaser = -1; g->n_pi = 0; g->chase_plies = 0;
    }

    /* threats made by this move */
    if (g->track_features && !battle) {
        int nb[4], nn = neighbours(to, nb);
        for (int i = 0; i < nn; ++i) {
            int Z = g->board[nb[i]];
            if (Z >= 0 && owner_of(Z) != P) set_bit(&g->f_threat[X], idx_rank_or_hidden(g, Z));
        }
    }

    memmove(&g->hist[1], &g->hist[0], (OR_HIST - 1) * sizeof(uint16_t));
    g->hist[0] = (uint16_t)action;
}

static int flag_dead(const or_game* g, int side)
{
    for (int p = side * 40; p < side * 40 + 40; ++p)
        if (g->type[p] == T_FLAG && !g->alive[p]) return 1;
    return 0;
}

int or_terminal_after(const or_game* g, int* winner)
{
    int Q = g->ply & 1, P = 1 - Q;
    int mv[400];
    *winner = -1;
    if (flag_dead(g, Q)) { *winner = P; return END_FLAG; }
    if (or_legal_moves(g, Q, mv) == 0) {
        if (or_physical_moves(g, P, mv) == 0) return END_NEITHER_CAN_MOVE;
        *winner = P;
        return END_NO_MOVES;
    }
    if (g->battleless >= g->rules.battleless_limit) return END_K_RULE;
    if (g->ply >= g->rules.max_plies) return END_CAP;
    return END_NONE;
}

int or_start_check(const or_game* g, int* winner)
{
    int P = g->ply & 1;
    int mv[400];
    *winner = -1;
    if (or_legal_moves(g, P, mv) > 0) return END_NONE;
    if (or_physical_moves(g, 1 - P, mv) == 0) return END_NEITHER_CAN_MOVE;
    *winner = 1 - P;
    return END_NO_MOVES;
}

uint64_t or_perft(const or_game* g, int depth, int use_brute)
{
    if (depth == 0) return 1;
    int mv[400];
    int P = g->ply & 1;
    int n;
    if (use_brute) {
        /* brute enumerator for the geometry, the same rule filters on top */
        int raw[400];
        int nr = or_brute_moves(g, P, raw);
        n = 0;
        for (int i = 0; i < nr; ++i) {
            int f = raw[i] / 100, t = raw[i] % 100;
            if (two_square_blocks(g, P, f, t) || chase_blocks(g, P, f, t)) continue;
            mv[n++] = raw[i];
        }
    } else {
        n = or_legal_moves(g, P, mv);
    }
    if (depth == 1) return (uint64_t)n;
    uint64_t total = 0;
    or_game* child = (or_game*)malloc(sizeof(or_game));
    for (int i = 0; i < n; ++i) {
        memcpy(child, g, sizeof(or_game));
        child->track_features = 0;
        or_apply(child, mv[i]);
        int w;
        /* an ended game has no continuation */
        if (or_terminal_after(child, &w) != END_NONE) continue;
        total += or_perft(child, depth - 1, use_brute);
    }
    free(child);
    return total;
}

/* ---------------------------------------------------------------- snapshot
 * Layout of the 784-byte position (little endian):
 *   0   type[80]      160 flags[80] (bit0 alive, bit1 revealed, bit2 moved,
 *   80  square[80]        bit3 scout-known, bits 4-6 cause of death)
 *   240 int16 ply     242 int16 battleless   244 last_battle  245 chaser (0xFF none)
 *   246 chase_plies   247 zero               248 ts_pid[2] (0xFF none)
 *   250 ts_len[2]     252 ts_sq[2][4] (0xFF unused)   260-271 zero
 *   272 uint16 hist[256] (move played i+1 plies ago, 0xFFFF none)
 */
void or_export(const or_game* g, uint8_t out[OR_POS_BYTES])
{
    memset(out, 0, OR_POS_BYTES);
    for (int p = 0; p < OR_NPIECE; ++p) {
        out[p] = g->type[p];
        out[80 + p] = g->sq[p];
        out[160 + p] = (uint8_t)(g->alive[p] | (g->revealed[p] << 1) | (g->moved[p] << 2) |
                                 (g->scout_known[p] << 3) | (g->cause[p] << 4));
    }
    out[240] = (uint8_t)(g->ply & 0xFF); out[241] = (uint8_t)(g->ply >> 8);
    out[242] = (uint8_t)(g->battleless & 0xFF); out[243] = (uint8_t)(g->battleless >> 8);
    out[244] = (uint8_t)g->last_battle;
    out[245] = g->chaser < 0 ? 0xFF : (uint8_t)g->chaser;
    out[246] = (uint8_t)g->chase_plies;
    for (int p = 0; p < 2; ++p) {
        out[248 + p] = g->ts_pid[p] < 0 ? 0xFF : (uint8_t)g->ts_pid[p];
        out[250 + p] = (uint8_t)g->ts_len[p];
        for (int i = 0; i < 4; ++i)
            out[252 + 4 * p + i] = (i < g->ts_len[p]) ? (uint8_t)g->ts_sq[p][i] : 0xFF;
    }
    for (int i = 0; i < OR_HIST; ++i) {
        out[272 + 2 * i] = (uint8_t)(g->hist[i] & 0xFF);
        out[273 + 2 * i] = (uint8_t)(g->hist[i] >> 8);
    }
}

int or_import(or_game* g, const uint8_t in[OR_POS_BYTES], const or_rules* rules, int track_features)
{
    uint8_t types[OR_NPIECE];
    for (int p = 0; p < OR_NPIECE; ++p) types[p] = in[p];
    or_game_init(g, types, rules, track_features);
    int count[2][T_NTYPES] = { { 0 } };
    for (int p = 0; p < OR_NPIECE; ++p) {
        if (types[p] >= T_NTYPES) return -1;
        count[p / 40][types[p]]++;
        uint8_t f = in[160 + p];
        g->sq[p] = in[80 + p];
        if (g->sq[p] >= OR_NSQ || or_is_lake(g->sq[p])) return -2;
        g->alive[p] = f & 1;
        g->revealed[p] = (f >> 1) & 1;
        g->moved[p] = (f >> 2) & 1;
        g->scout_known[p] = (f >> 3) & 1;
        g->cause[p] = (f >> 4) & 7;
        if (g->alive[p] && g->cause[p]) return -3;
    }
    for (int s = 0; s < 2; ++s)
        for (int t = 0; t < T_NTYPES; ++t)
            if (count[s][t] != TYPE_COUNT[t]) return -4;
    for (int s = 0; s < OR_NSQ; ++s) g->board[s] = or_is_lake(s) ? -2 : -1;
    for (int p = 0; p < OR_NPIECE; ++p) {
        if (!g->alive[p]) continue;
        if (g->board[g->sq[p]] != -1) return -5;
        g->board[g->sq[p]] = p;
    }
    g->ply = (int)(int16_t)(in[240] | (in[241] << 8));
    g->battleless = (int)(int16_t)(in[242] | (in[243] << 8));
    if (g->ply < 0 || g->battleless < 0 || g->battleless > g->ply) return -6;
    g->last_battle = in[244] ? 1 : 0;
    g->chaser = in[245] == 0xFF ? -1 : in[245];
    g->chase_plies = in[246];
    if (g->chaser > 1) return -7;
    for (int p = 0; p < 2; ++p) {
        g->ts_pid[p] = in[248 + p] == 0xFF ? -1 : in[248 + p];
        g->ts_len[p] = in[250 + p];
        for (int i = 0; i < 4; ++i) g->ts_sq[p][i] = in[252 + 4 * p + i] == 0xFF ? -1 : in[252 + 4 * p + i];
        if (g->ts_pid[p] >= 0 && (g->ts_pid[p] >= OR_NPIECE || g->ts_len[p] < 2 || g->ts_len[p] > 4)) return -8;
        if (g->ts_pid[p] < 0 && g->ts_len[p] != 0) return -8;
        /* the squares of the piece's last moves lie on the board */
        for (int i = 0; i < g->ts_len[p] && i < 4; ++i)
            if (g->ts_sq[p][i] < 0 || g->ts_sq[p][i] >= OR_NSQ || or_is_lake(g->ts_sq[p][i])) return -8;
    }
    for (int i = 0; i < OR_HIST; ++i) g->hist[i] = (uint16_t)(in[272 + 2 * i] | (in[273 + 2 * i] << 8));
    /* chase positions: undo the chase plies from the current board */
    if (g->chaser >= 0) {
        if (g->chase_plies < 1 || g->chase_plies > OR_HIST) return -9;
        int b[OR_NSQ];
        memcpy(b, g->board, sizeof(b));
        uint8_t tmp[OR_MAX_PI][OR_NSQ];
        int nt = 0;
        for (int i = 0; i < g->chase_plies; ++i) {
            int mover = (g->ply - 1 - i) & 1;
            if (g->hist[i] == 0xFFFF) return -10;
            if (mover == g->chaser) {
                if (nt >= OR_MAX_PI) return -11;
                for (int s = 0; s < OR_NSQ; ++s) tmp[nt][s] = b[s] >= 0 ? (uint8_t)b[s] : 0xFF;
                nt++;
            }
            int f = g->hist[i] / 100, t = g->hist[i] % 100;
            if (f >= OR_NSQ || b[t] < 0 || b[f] != -1) return -12;
            b[f] = b[t];
            b[t] = -1;
        }
        g->n_pi = nt;
        for (int i = 0; i < nt; ++i) memcpy(g->pi[i], tmp[nt - 1 - i], OR_NSQ);
    } else if (g->chase_plies != 0) {
        return -13;
    }
    return 0;
}
