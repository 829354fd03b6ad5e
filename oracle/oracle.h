/*
 * Stratego oracle: plain, single-threaded C restatement of the game engine,
 * the observation planes, the belief sampler and the random rollouts.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * includes anything in this directory; only the test suite, the package's
 * smoke check and the benchmark's CPU baseline leg load it.  It shares no
 * code, header, table or constant generator with the CUDA path.
 *
 * Sources (arXiv 2511.07312, "Superhuman AI for Stratego Using Self-Play
 * Reinforcement Learning and Test-Time Search"):
 *   App. A "Rules of Stratego"          board, pieces, movement, battles,
 *                                        two-square and continuous-chasing
 *                                        rules (Tab. pieces, Tab. chase)
 *   App. B.1-B.4                        simulator state machines, reset to
 *                                        non-initial states
 *   App. C.1-C.2                        information-state channels
 *   App. D.1 (Tab. game-hyper)          k-move rule and game-length cap
 *   App. E "Search"                     belief samples, rollouts, the search
 *                                        update (search.c)
 *   Salmon et al., SC'11                Philox4x32-10
 *
 * Readings where the paper is silent are listed at the top of each source
 * file and repeated in the design notes.
 */
#ifndef STRATEGO_ORACLE_H
#define STRATEGO_ORACLE_H

#include <stdint.h>
#include <stddef.h>

#define OR_NPIECE      80      /* 40 per side: red pids 0-39, blue pids 40-79 */
#define OR_NSQ         100     /* square s = 10*row + col, row 0 = red's back row */
#define OR_MASK_BYTES  1264    /* 10,000 mask bits padded to a 16-byte multiple */
#define OR_NCHAN       487     /* observation channels (App. C) */
#define OR_HIST        256     /* moves of history kept in a position snapshot */
#define OR_MAX_PI      160     /* stored chase positions (<= ceil(k/2) for k <= 255) */
#define OR_POS_BYTES   784     /* size of the position snapshot layout */
#define OR_SEARCH_MAX_MOVES 256 /* legal moves of one side never exceed 244 */

/* Type codes follow the order of channels 0-11 (App. C.1). */
enum { T_SPY = 0, T_SCOUT = 1, T_MINER = 2, T_SERGEANT = 3, T_LIEUTENANT = 4,
       T_CAPTAIN = 5, T_MAJOR = 6, T_COLONEL = 7, T_GENERAL = 8, T_MARSHAL = 9,
       T_FLAG = 10, T_BOMB = 11, T_NTYPES = 12 };

/* Ending codes. */
enum { END_NONE = 0, END_FLAG = 1, END_NO_MOVES = 2, END_NEITHER_CAN_MOVE = 3,
       END_K_RULE = 4, END_CAP = 5 };

/* Rule toggles. */
#define OR_RULE_TWO_SQUARE 1
#define OR_RULE_CHASE      2
/* Rollout policy: the magnet policy instead of uniform over the legal moves
 * (rollouts and search only; the game rules ignore it). */
#define OR_ROLLOUT_MAGNET  0x100

typedef struct {
    int battleless_limit;   /* k of the k-move rule (App. D.1: 100 in training) */
    int max_plies;          /* draw once this many plies have been played */
    int flags;              /* OR_RULE_* */
} or_rules;

typedef struct {
    /* per piece id */
    uint8_t type[OR_NPIECE];
    uint8_t sq[OR_NPIECE];        /* square while alive; battle square once dead */
    uint8_t alive[OR_NPIECE];
    uint8_t revealed[OR_NPIECE];
    uint8_t moved[OR_NPIECE];
    uint8_t scout_known[OR_NPIECE];
    uint8_t cause[OR_NPIECE];     /* cause of death 1-6, 0 while alive */
    int board[OR_NSQ];            /* piece id, -1 empty, -2 lake */
    int ply;                      /* plies played in this game */
    int battleless;               /* consecutive plies without a battle */
    int last_battle;              /* the previous ply was a battle */
    /* two-square rule: last-moved piece of each player and its last squares */
    int ts_pid[2];
    int ts_len[2];
    int ts_sq[2][4];
    /* continuous chasing */
    int chaser;                   /* -1 none */
    int chase_plies;              /* plies since the chase began */
    int n_pi;
    uint8_t pi[OR_MAX_PI][OR_NSQ];/* boards (piece id per square, 0xFF empty) after chaser threats */
    /* history: hist[i] = move played i+1 plies ago (from*100+to), 0xFFFF none */
    uint16_t hist[OR_HIST];
    /* sticky per-piece features (App. C.1) */
    uint32_t f_threat[OR_NPIECE];   /* bits 0-9 revealed type, 10 hidden */
    uint32_t f_evade[OR_NPIECE];    /* same */
    uint32_t f_active[OR_NPIECE];   /* same */
    uint32_t f_prot[OR_NPIECE];     /* 0-10 revealed Spy..Marshal,Bomb; 11 empty; 12 hidden */
    uint32_t f_pagainst[OR_NPIECE]; /* 0-10 revealed type, 11 hidden */
    uint32_t f_pby[OR_NPIECE];      /* 0-10 revealed type, 11 hidden */
    uint32_t f_pbyagainst[OR_NPIECE];
    int track_features;
    or_rules rules;
} or_game;

/* ---- philox.c ---- */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
uint32_t or_uniform(uint32_t r, uint32_t n);   /* floor(r * n / 2^32) */

/* ---- rules.c ---- */
int  or_is_lake(int s);
int  or_battle(int attacker_type, int defender_type);   /* 1 attacker wins, 2 defender wins, 3 tie */
void or_setup_types(uint64_t seed, uint32_t slot, uint32_t episode, uint8_t types[OR_NPIECE]);
void or_game_init(or_game* g, const uint8_t types[OR_NPIECE], const or_rules* rules, int track_features);
int  or_physical_moves(const or_game* g, int player, int* moves);       /* returns count, moves = from*100+to */
int  or_legal_moves(const or_game* g, int player, int* moves);          /* full rules */
int  or_move_legal(const or_game* g, int player, int action);
void or_apply(or_game* g, int action);
int  or_terminal_after(const or_game* g, int* winner);                   /* ending code after the last ply */
int  or_start_check(const or_game* g, int* winner);                      /* acting player cannot move */
void or_mask_from_moves(const int* moves, int n, uint8_t mask[OR_MASK_BYTES]);
int  or_two_square_applies(const or_game* g);
int  or_brute_moves(const or_game* g, int player, int* moves);           /* independent enumerator */
uint64_t or_perft(const or_game* g, int depth, int use_brute);
void or_export(const or_game* g, uint8_t out[OR_POS_BYTES]);
int  or_import(or_game* g, const uint8_t in[OR_POS_BYTES], const or_rules* rules, int track_features);

/* ---- obs.c ---- */
void or_encode_planes(const or_game* g, int player, uint8_t* planes_u8, uint16_t* planes_bf16);
uint16_t or_bf16_ratio(uint32_t num, uint32_t den);
uint8_t  or_u8_ratio(uint32_t num, uint32_t den);
void or_side_marginals(const or_game* g, int side, uint32_t* num /*[40][12]*/, uint32_t* den /*[40][12]*/);

/* ---- policy.c ---- */
/* The rollout policy's move from the legal moves in ascending order and the
 * ply's four Philox words (magnet != 0: the magnet policy). */
int or_policy_pick(const int* moves, int n, const uint32_t w[4], int magnet);

/* ---- belief.c ---- */
void or_belief_sample_one(const or_game* g, uint64_t seed, uint32_t stream, uint32_t sample,
                          uint8_t out_types[40]);

/* App. E search (search.c): per-candidate-move rollouts and the tabular
 * magnetic-mirror-descent update; outputs [P][OR_SEARCH_MAX_MOVES](x4). */
int orx_search(const uint8_t* pos, int P, int S, int depth, uint64_t seed, const uint32_t* stream_ids,
               const float* pi_theta, const float* q_given, double alpha, double beta, int k, int cap, int flags,
               int32_t* n_moves, int16_t* actions, int32_t* tallies, double* q, double* pi, int16_t* chosen,
               uint8_t* status);

#endif
