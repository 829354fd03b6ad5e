/*
 * stratego.h -- C ABI of the GB300 Stratego engine.
 *
 * A batched, GPU-resident implementation of the game engine that self-play
 * and test-time search of arXiv 2511.07312 ("Superhuman AI for Stratego
 * Using Self-Play Reinforcement Learning and Test-Time Search") spend their
 * non-network time in: legal-move masks, move apply and battles, endings with
 * auto-reset, observation planes, belief samples of the opponent's hidden
 * pieces, fixed-depth rollouts, the per-move search with its policy update,
 * queries about past steps, and serving.  Section references are to that
 * paper: App. A (rules), App. B (simulator), App. C (information state),
 * App. D.1 (game-rule hyperparameters), App. E (search).
 *
 * Conventions shared by every entry point
 *  - Square s = 10*row + col, row 0 is red's back row, col 0 is file a.
 *    Lakes: 42,43,52,53,46,47,56,57 (App. A: 92 occupiable squares).
 *  - Piece ids: red 0-39 start on squares 0-39, blue 40-79 on squares 60-99.
 *  - Type codes 0-11: Spy, Scout, Miner, Sergeant, Lieutenant, Captain,
 *    Major, Colonel, General, Marshal, Flag, Bomb (the order of App. C
 *    channels 0-11).
 *  - Action a = from*100 + to.  A legal-action mask is 1264 bytes: bit a&7 of
 *    byte a>>3, bytes 1250-1263 zero.
 *  - Red (player 0) moves on even plies.
 *  - Ending codes: 0 none, 1 flag captured, 2 the player to move has no legal
 *    move (the other player wins), 3 neither player can move (draw), 4 k
 *    battleless plies (draw), 5 game-length cap (draw).  Rewards are from the
 *    red player's view: +1, -1, or 0 (App. B.1, ComputeRewardPl0).
 *  - Random numbers: Philox4x32-10 (Salmon et al., SC'11) keyed by the 64-bit
 *    seed (low word first); the counter layout of each draw is given at the
 *    entry point that makes it.  A uniform draw in [0,n) is floor(r*n/2^32).
 *
 * Memory and streams
 *  - Every array argument is a caller-owned DEVICE pointer unless the
 *    comment says HOST.  The library never frees caller memory.
 *  - Calls are asynchronous on the given stream (cudaStream_t passed as
 *    void*, NULL = legacy default stream).  The caller keeps inputs alive and
 *    unmodified until the work completes.
 *  - An st_env owns its device state (allocated once in st_env_create, App.
 *    B "no dynamic allocation after construction") and its stream.
 *
 * Errors
 *  - Every call returns st_status.  Argument errors are detected on the host
 *    before anything is enqueued (ST_ERR_INVALID, nothing changes).
 *  - st_last_error() returns a thread-local description of the last failure.
 *  - Errors found on the device (an illegal supplied action, an invalid
 *    snapshot) never fault: the item is left unchanged and the error is
 *    latched; st_env_sync() reports it for an env, per-item status arrays
 *    report it for the stateless calls.
 */
#ifndef STRATEGO_GB300_H
#define STRATEGO_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum st_status {
    ST_OK = 0,
    ST_ERR_INVALID = 1,          /* bad argument; nothing was enqueued */
    ST_ERR_OOM = 2,              /* device allocation failed at create time */
    ST_ERR_CUDA = 3,             /* a CUDA runtime call failed */
    ST_ERR_ILLEGAL_ACTION = 4,   /* a supplied action was not legal (latched) */
    ST_ERR_TIMEOUT = 5,          /* a bounded wait expired */
    ST_ERR_BUSY = 6,             /* no capacity right now; retry later */
    ST_ERR_NOT_READY = 7,        /* result not available yet */
    ST_ERR_BAD_POSITION = 8      /* a snapshot or log failed validation (latched) */
} st_status;

/* Rule flags (App. A "Additional rules for competitive play"). */
#define ST_RULE_TWO_SQUARE 1u    /* two-square rule, App. A and App. B.2 */
#define ST_RULE_CHASE      2u    /* continuous-chasing rule, Tab. chase, App. B.3 */
#define ST_AUTORESET       4u    /* env only: ended games restart at once (App. B.1) */
#define ST_RULES_ALL       (ST_RULE_TWO_SQUARE | ST_RULE_CHASE)
/* Rollout policy (st_rollout, st_search, the server; refused by the env and
 * the observation calls): the magnet policy rho of Tab. notation -- a piece
 * with a legal move uniformly (ascending squares, word 0 of the ply's Philox
 * counter), then one of its legal moves uniformly (ascending actions, word
 * 1) -- instead of uniform over the legal moves (word 0). */
#define ST_ROLLOUT_MAGNET  0x100u

#define ST_MASK_BYTES   1264
#define ST_NCHAN        487      /* observation channels, App. C */
#define ST_MAX_GAMES    (1 << 22)
#define ST_MAX_BATTLELESS 255

/* Game-rule parameters (App. D.1, Tab. game-hyper). */
typedef struct st_rules {
    int16_t battleless_limit;    /* k of the k-move rule: 1..255 (paper: 100 training, 200 online) */
    int16_t max_plies;           /* draw after this many plies: 1..32767 (paper: 4000) */
    uint32_t flags;              /* ST_RULE_* */
} st_rules;

/*
 * Position snapshot: everything needed to continue a game exactly (App. B.4
 * "reset to a non-initial state"), 784 bytes, little endian.
 *   flags[p]: bit0 alive, bit1 revealed (a battle showed the type), bit2 has
 *   moved, bit3 moved more than one square once (so it is a Scout), bits4-6
 *   cause of death 1-6 (App. C.1 "Causes of death"), 0 while alive.
 *   square[p]: current square, or the battle square of a captured piece.
 *   last_battle: the previous ply was a battle.
 *   chaser: player whose continuous chase is in progress (0xFF none);
 *   chase_plies: plies since that chase began (its moves are hist[0..n-1]).
 *   ts_*: two-square rule state per player -- last-moved piece, number of
 *   squares recorded (2-4) and those squares, oldest first (0xFF unused).
 *   hist[i]: the action played i+1 plies ago, 0xFFFF if unknown.
 */
typedef struct st_position {
    uint8_t type[80];
    uint8_t square[80];
    uint8_t flags[80];
    int16_t ply;
    int16_t battleless;
    uint8_t last_battle;
    uint8_t chaser;
    uint8_t chase_plies;
    uint8_t reserved0;            /* zero */
    uint8_t ts_pid[2];
    uint8_t ts_len[2];
    uint8_t ts_sq[2][4];
    uint8_t reserved1[12];        /* zero */
    uint16_t hist[256];
} st_position;

typedef struct st_env st_env;

typedef struct st_env_config {
    int32_t num_games;            /* parallel game slots N, 1..ST_MAX_GAMES */
    uint64_t seed;                /* Philox key */
    st_rules rules;
    uint32_t env_flags;           /* ST_AUTORESET */
    int32_t device;               /* CUDA device ordinal */
    void* stream;                 /* cudaStream_t for every call on this env; NULL = default */
} st_env_config;

/* Library identification and the thread-local text of the last error. */
const char* st_version(void);
const char* st_last_error(void);

/*
 * st_env_create: allocate the env's device state for cfg->num_games slots
 * and start every slot's first game (episode 0).  Setup of slot i, episode e
 * (App. A: 40 pieces on each side's four back rows): each side's sorted
 * 40-piece multiset is Fisher-Yates shuffled, i = 39..1, j = U[0,i+1) from
 * draw d = 39-i, word d%4 of Philox at counter (i, e, 0, 1<<24 | side<<8 | d/4),
 * and laid on the side's squares in ascending order.
 * Errors: ST_ERR_INVALID (bad config), ST_ERR_OOM, ST_ERR_CUDA.
 */
st_status st_env_create(const st_env_config* cfg, st_env** out);

/* Release every device allocation of the env (synchronizes its stream). */
st_status st_env_destroy(st_env* env);

/*
 * st_env_reset: start a new game in the slots with which[i] != 0 (all slots
 * if which is NULL).  Each restarted slot's episode counter is incremented.
 * setups: [N][80] type per piece id, or NULL for the Philox setup above.
 * A setup whose type counts per side differ from Tab. pieces leaves the slot
 * unchanged and latches ST_ERR_BAD_POSITION.
 */
st_status st_env_reset(st_env* env, const uint8_t* setups, const uint8_t* which);

/*
 * st_env_step: one ply in every slot (App. B.1 ApplyActions and
 * SampleRandomLegalAction).  actions[N] int16: the action for each slot, or
 * -1 for the uniform random policy; NULL = random everywhere.  The random
 * policy at ply t of episode e in slot i takes word 0 of Philox at counter
 * (i, e, t, 2<<24) and plays the floor(r*n/2^32)-th of the n legal actions in
 * ascending order.  After the ply, endings are checked in ending-code order;
 * with ST_AUTORESET an ended game restarts at once.
 * Outputs (each may be NULL), per slot:
 *   action_out[N] int16  action played (-1 if none was played)
 *   reward_out[N] int8   red-player reward of a game that ended on this ply
 *   done_out[N]   uint8  ending code
 *   ply_out[N]    int16  ply index of the action in its game
 *   mask_out[N][1264]    legal mask of the player to move afterwards (of the
 *                        new game after an auto-reset; zero for an ended game
 *                        without auto-reset)
 * A slot whose supplied action is illegal is left unchanged (action_out -1,
 * mask of the unchanged state) and ST_ERR_ILLEGAL_ACTION is latched.
 */
st_status st_env_step(st_env* env, const int16_t* actions, int16_t* action_out, int8_t* reward_out,
                      uint8_t* done_out, int16_t* ply_out, uint8_t* mask_out);

/* The random policy's action for every slot at the current state, without
 * playing it: actions[N] int16 (device), the action st_env_step with
 * actions NULL would play next, -1 for an ended game or a player without a
 * legal move (App. B.1 SampleRandomLegalAction). */
st_status st_env_sample_actions(st_env* env, int16_t* actions);

/*
 * st_env_run: n_steps random-policy plies in every slot in one persistent
 * launch, game state held on chip between plies.  Step j of the call writes
 * the outputs of st_env_step into ring row j % ring_steps of each output
 * ([ring_steps][N] and [ring_steps][N][1264]); any output may be NULL.
 * Results are identical to n_steps calls of st_env_step with actions NULL.
 * When the slots outnumber the games resident on the GPU and 512 <= n_steps <= 32768,
 * each slot's plies may run as 2 to 4 parts of >= 256 plies, claimed as
 * separate work units so that the launch's last wave is nearly full (a part
 * waits, with a bound of a few seconds, for the slot's previous part to be
 * stored; running out latches ST_ERR_TIMEOUT for the slot).
 */
st_status st_env_run(st_env* env, int32_t n_steps, int32_t ring_steps, int16_t* action_ring,
                     int8_t* reward_ring, uint8_t* done_ring, int16_t* ply_ring, uint8_t* mask_ring);

/* Launch shape of st_env_run: warps per block (1..8), blocks per SM (0 =
 * occupancy maximum), games a warp steps side by side (1, 2, 4 or 8: teams
 * of 32, 16, 8 or 4 lanes) and slots each team claims per queue fetch (>=1).
 * Results do not depend on the shape. */
st_status st_env_set_launch(st_env* env, int32_t warps_per_block, int32_t blocks_per_sm, int32_t games_per_warp,
                            int32_t games_per_fetch);

/* The launch shape st_env_run uses now, as four int32 values: warps per
 * block, blocks per SM (the request of st_env_set_launch clamped to what
 * fits on an SM, or that maximum for a request of 0), games per warp and
 * slots per fetch.  out: host memory owned by the caller. */
st_status st_env_get_launch(st_env* env, int32_t* out);

/* Wait for the env's stream; return and clear a latched device error. */
st_status st_env_sync(st_env* env);

/* Per-slot counters [N][8] uint32: games ended with codes 1-5, plies played,
 * red wins, blue wins (cumulative since create). */
st_status st_env_stats(st_env* env, uint32_t* stats_out);

/* Snapshots of slots idx[0..n-1] (App. B.4).  Export writes out[n]; import
 * replaces the slots' games (episode counters unchanged).  An invalid
 * snapshot leaves its slot unchanged and latches ST_ERR_BAD_POSITION. */
st_status st_env_export(st_env* env, const int32_t* idx, int32_t n, st_position* out);
st_status st_env_import(st_env* env, const int32_t* idx, int32_t n, const st_position* in);

#define ST_POOL_MIRROR   1u          /* st_env_set_setup_pool: left-right orientation randomisation */
#define ST_MAX_POOL      (1 << 20)   /* setups per side in a pool */

/*
 * st_env_set_setup_pool: new games (auto-reset, and st_env_reset without
 * setups) take each side's setup from a pool of pre-generated setups (Sec.
 * "Data Collection": a pool per player; App. "Learned Setups": left-right
 * orientation randomisation).  Side s of the game of slot g at episode e
 * takes entry uniform_below(w0, M) of pool[s], (w0, w1, w2, w3) being Philox
 * at counter (g, e, 0, 7<<24 | s); with ST_POOL_MIRROR the entry is mirrored
 * left-right (file a <-> j) when w1 is odd.
 *   pool: device, [2][M][40] uint8: per side and entry, the types on the
 *         side's 40 setup squares in ascending square order (red 0-39, blue
 *         60-99); copied into the env (the caller keeps ownership).  M = 0
 *         turns the pool off.
 * Errors (nothing changes): ST_ERR_INVALID for M outside [0, ST_MAX_POOL],
 * unknown flags, a NULL pool with M > 0, or an entry that is not one side's
 * 40 pieces.  Synchronous: the pool is checked on the host.
 */
st_status st_env_set_setup_pool(st_env* env, const uint8_t* pool, int32_t M, uint32_t flags);

/*
 * st_env_pin: restarts from a fixed non-initial position (App. B.4, for
 * search; the snapshot's history, two-square and chase state come with it,
 * App. B.3).  From now on slot idx[i] restarts from states[i] whenever its
 * game ends (auto-reset) and at st_env_reset without setups, its episode
 * counter incremented as for any new game; games in progress continue.  Each
 * call replaces the whole pin set (n = 0 clears it); with a slot listed
 * twice the later entry wins.  Slots not pinned restart from the pool or
 * the Philox setup.
 *   idx[n] int32, states[n]: device, caller-owned, read in stream order.
 * Errors: ST_ERR_INVALID for n outside [0, N] or NULL arrays with n > 0
 * (nothing changes); a slot index outside [0, N) or an invalid snapshot
 * leaves that entry unpinned and latches ST_ERR_BAD_POSITION.
 */
st_status st_env_pin(st_env* env, const int32_t* idx, int32_t n, const st_position* states);

#define ST_MAX_HISTORY 32767          /* steps kept by the history ring */

/*
 * History (App. B.1: the simulator doubles as the rollout buffer and
 * answers queries about past time steps from a circular buffer).  A time
 * step t counts env steps: st_env_step adds 1, st_env_run n_steps; the
 * state at step t is every slot's state after t steps, before step t's ply.
 * st_env_enable_history(H) keeps, per slot, one 4-byte record of each of
 * the last H steps (action, ending code, red's reward, whether the step's
 * state began a game): H x N x 4 bytes of device memory; H = 0 turns it off.
 * Steps taken while it is off are not recorded; games in progress when it
 * is turned on after steps were taken count as begun before the window.
 * Past positions are rebuilt by replaying a game's recorded actions from
 * its start (recompute rather than store, App. B.1), so a query about step
 * t is answered for t in the window [max(first recorded step, now - H),
 * now], and a slot's position only if its game began inside the window,
 * as a new game (Philox setup, pool or pin) under the reset sources still
 * in force.  Errors: ST_ERR_INVALID for t outside the window or a NULL
 * output (nothing is enqueued); ST_ERR_OOM if the ring does not fit.
 */
st_status st_env_enable_history(st_env* env, int32_t H);

/* Steps taken since create (App. B.1 CurrentStep). */
st_status st_env_current_step(st_env* env, int64_t* now);

/*
 * Positions at step t (the state every historical query of App. B.1 is
 * about: acting player = ply & 1, moves played = ply, moves since the last
 * attack = battleless, unknown pieces and piece types from the flags and
 * types; legal masks via st_positions_mask).  out[N]: snapshots (device).
 * status[N] (may be NULL): 0 rebuilt, 2 the game began before the window
 * or before the last change of the setup pool or pins, 3 it began from
 * given setups or an import (out is then left unwritten; step t = now is
 * always answered).  ended[N]: ending code of the slot's game if it was
 * over at step t, else 0; since[N]: steps since the step that ended it
 * (GetTerminatedSince; 0 while running, -1 if that step left the window).
 */
st_status st_env_history_positions(st_env* env, int64_t t, st_position* out, uint8_t* status, uint8_t* ended,
                                   int32_t* since);

/* The record of step t < now per slot (any output may be NULL): action
 * played (-1 none; GetPlayedActions), ending code reported (1 flag captured,
 * ...), red's reward (ComputeRewardPl0), and 0 or how the step's state began
 * a game (1 new game, 2 given setups, 3 import). */
st_status st_env_history_steps(st_env* env, int64_t t, int16_t* action, uint8_t* done, int8_t* reward,
                               uint8_t* start);

/* The setup and action log of each slot's game at step t, the input of
 * st_obs_encode (game g, ply plies[g]) for its planes and mask at step t
 * (ComputeInfostateTensor): setups[N][80], logs[N][L] (-1 after the last
 * action), plies[N]; status[N] as for positions, plus 4 a pinned start (no
 * setup to replay from) and 5 more than L actions. */
st_status st_env_history_logs(st_env* env, int64_t t, int32_t L, uint8_t* setups, int16_t* logs, int16_t* plies,
                              uint8_t* status);

/*
 * Replay of action logs (App. B.1: states are reconstructed on demand from
 * compact records).  Game g < num_logs starts from setups[g] (type per piece
 * id, [num_logs][80]) and plays actions[g][0..log_len-1] ([num_logs][log_len]
 * int16); item b is game[b] after ply[b] plies.  Every logged action is
 * checked for legality and no intermediate position may have ended the game.
 * Items sorted by (game, ply) are cheapest: a warp walks consecutive items of
 * one game once.  item_status[B] (may be NULL): 0 ok, 1 out-of-range item,
 * bad setup or illegal log entry (its outputs are zero).
 */
st_status st_replay_positions(const uint8_t* setups, const int16_t* actions, int32_t log_len, int32_t num_logs,
                              const int32_t* game, const int16_t* ply, int32_t B, const st_rules* rules,
                              st_position* out, uint8_t* item_status, void* stream);

/* Consecutive items a replay block takes (default 32); a process-wide
 * tuning knob. */
st_status st_replay_set_chunk(int32_t items_per_block);

/*
 * st_obs_encode: observation planes of App. C for B replayed items, for the
 * player player[b] (0/1) or the player to move (-1 or player NULL), in the
 * absolute board frame.  planes [B][487][100] uint8: indicators 0/1, history
 * -1 as 255, probabilities and fractions num/den as floor(255*num/den+1/2);
 * planes_bf16 [B][487][100] bf16 bits: the same values with num/den rounded
 * to nearest-even bf16; mask [B][1264]: legal mask of the player to move.
 * Any output may be NULL.
 */
st_status st_obs_encode(const uint8_t* setups, const int16_t* actions, int32_t log_len, int32_t num_logs,
                        const int32_t* game, const int16_t* ply, const int8_t* player, int32_t B,
                        const st_rules* rules, uint8_t* planes, uint16_t* planes_bf16, uint8_t* mask,
                        uint8_t* item_status, void* stream);

/*
 * st_obs_encode_static: st_obs_encode for callers that cannot allocate
 * device memory while they run -- for example a serving or training loop
 * that fixes its memory budget at start-up and must not call the allocator
 * afterwards, or a caller running under a custom memory manager that does
 * not see stream-ordered allocations.  (The paper has no counterpart of
 * this entry point.)
 *
 * Same arguments, outputs and errors as st_obs_encode; the per-item replay
 * records that st_obs_encode allocates per call (about 1.6 KB per item) live
 * instead in a fixed array inside this library's device image, sized for
 * ST_OBS_STATIC_MAX_ITEMS items (about 6.7 MB).  Every GPU on which the
 * library is loaded holds that array until the process exits.
 *  - B > ST_OBS_STATIC_MAX_ITEMS is rejected with ST_ERR_INVALID before
 *    anything is enqueued; split the batch or use st_obs_encode.
 *  - It never calls cudaMalloc, cudaFree, cudaMallocAsync or any other
 *    allocating routine.
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture on that device.  The address is kept for the
 *    life of the process: the entry point assumes the device's primary
 *    context (the one the CUDA runtime uses) throughout, and that
 *    cudaDeviceReset is not called on the device afterwards (a reset
 *    reloads the library's device image, and the kept address would be
 *    stale).
 *  - All calls share the one array: calls whose work overlaps on the GPU
 *    (different streams, or threads, without ordering between them) race
 *    and may corrupt each other's outputs.  Order them on one stream.
 *  - Each call writes every record it later reads, so what an earlier call
 *    left in the array never reaches an output.
 */
#define ST_OBS_STATIC_MAX_ITEMS 4096
st_status st_obs_encode_static(const uint8_t* setups, const int16_t* actions, int32_t log_len, int32_t num_logs,
                               const int32_t* game, const int16_t* ply, const int8_t* player, int32_t B,
                               const st_rules* rules, uint8_t* planes, uint16_t* planes_bf16, uint8_t* mask,
                               uint8_t* item_status, void* stream);

/*
 * st_belief_sample: K assignments of types to the hidden pieces of the
 * opponent of the player to move in each position, uniform over the
 * assignments consistent with the public history (App. E step 1, with the
 * uniform posterior standing in for the belief network): revealed and
 * captured pieces keep their type, a piece that moved more than one square is
 * a Scout, a moved piece is neither Bomb nor Flag, type counts are respected.
 * Draw w of sample k of position p is word w%4 of Philox at counter
 * (stream_ids[p] or p, k, 0, 3<<24 | w/4); the immovable pieces are placed
 * by a partial Fisher-Yates over the unmoved hidden pieces in ascending
 * square order, the movable multiset by a full Fisher-Yates over the other
 * hidden pieces in ascending square order.
 * types[P][K][40]: type of opponent piece id 40*opp + i for i < 40.
 */
st_status st_belief_sample(const st_position* pos, int32_t P, int32_t K, uint64_t seed,
                           const uint32_t* stream_ids, uint8_t* types, uint8_t* item_status, void* stream);

/*
 * st_rollout: for each position and each of K samples, replace the hidden
 * opponent types by the sample (types, or the st_belief_sample draw when
 * types is NULL) and play up to `depth` plies of the rollout policy (uniform
 * over the legal moves, or the magnet policy when rules->flags has
 * ST_ROLLOUT_MAGNET), ply d drawing from Philox at counter (stream_ids[p] or
 * p, k, d, 4<<24) (App. E step 2 with a random policy in place of the move
 * network).  tallies[P][4]
 * int32: wins, losses, draws of the player to move at the root, and
 * rollouts unfinished after `depth` plies.
 */
st_status st_rollout(const st_position* pos, int32_t P, int32_t K, int32_t depth, uint64_t seed,
                     const uint32_t* stream_ids, const uint8_t* types, const st_rules* rules,
                     int32_t* tallies, uint8_t* item_status, void* stream);

/*
 * st_positions_mask: for each snapshot, the legal mask of the player to move
 * (App. B.1 ComputeLegalActionMask; the 1,264-byte layout of st_env_step),
 * its number of legal moves (GetHasLegalMovement: > 0), and whether the
 * two-square rule removes one of that player's moves (App. B.2,
 * ComputeTwoSquareRuleApplies; 0 when the rules leave it off).  Arrays are
 * device, caller-owned, [P] (mask [P][1264], 16-byte aligned); any output
 * may be NULL.  item_status[P]: 0 ok, 1 invalid snapshot (outputs zero).
 */
st_status st_positions_mask(const st_position* pos, int32_t P, const st_rules* rules, uint8_t* mask,
                            int32_t* n_legal, uint8_t* two_square, uint8_t* item_status, void* stream);

#define ST_SEARCH_MAX_MOVES 256   /* one side never has more than 244 legal moves */

/*
 * st_search: per-candidate-move search with the tabular magnetic-mirror-
 * descent update (App. E "Search", steps 1-4; Sec. "Test-Time Search via
 * Update Equivalence"), with the uniform belief sampler in place of the
 * belief network and the uniform (or, with ST_ROLLOUT_MAGNET, the magnet)
 * rollout policy in place of the move network.
 * For each position p, the player to move being the searcher:
 *   1. S configurations of the opponent's hidden pieces; configuration s is
 *      st_belief_sample's sample s of stream stream_ids[p] (p if NULL);
 *   2. one rollout per (legal move j in ascending action order,
 *      configuration s): move j, then up to depth-1 rollout-policy plies,
 *      ply d drawing from Philox at counter (stream, j*S + s, d, 5<<24);
 *   3. q[j] = mean over the S rollouts of +1 win, -1 loss, 0 draw or
 *      unfinished (for the searcher), 0 when S = 0; or, with q_values given,
 *      the given value of move j and no rollout (a value network's role);
 *   4. rho[j] = 1 / (pieces with a legal move * legal moves of move j's
 *      piece) (the magnet policy, Tab. notation); pi[j] proportional to
 *      exp((q[j] + alpha ln rho[j] + beta ln pi_theta[j]) / (alpha + beta)),
 *      in double; chosen = the first move whose ascending running sum of the
 *      unnormalized weights exceeds u * (their sum), u = (w0 >> 5) * 2^-27 +
 *      (w1 >> 6) * 2^-53 from Philox at counter (stream, 0, 0, 6<<24).
 * Arguments (device pointers, caller-owned; P <= 65535, S >= 0, depth >= 1,
 * alpha, beta >= 0 with alpha + beta > 0; App. E uses 0.002 and 0.02):
 *   pos[P]                     positions;
 *   pi_theta[P][10000] float   move-network probabilities by action (NULL:
 *                              uniform over the legal moves); only legal
 *                              entries are read, a zero excludes the move;
 *   q_values[P][10000] float   per-move values by action for the searcher
 *                              (NULL: from the rollouts); only legal entries
 *                              are read;
 *   n_moves[P] int32           the searcher's legal moves (0: none searched);
 *   actions[P][256] int16      those moves ascending, -1 after the last;
 *   tallies[P][256][4] int32   wins, losses, draws, unfinished per move;
 *   q, pi[P][256] double       values and the updated policy (0 after the last);
 *   chosen[P] int16            the move played, -1 when there is none;
 *   item_status[P] uint8       0 ok, 1 invalid position, 2 pi_theta zero on
 *                              every legal move (may be NULL).
 * Errors: ST_ERR_INVALID for bad sizes or coefficients or a NULL output,
 * before anything is enqueued.  Stream-ordered; scratch is stream-ordered
 * device memory.
 */
st_status st_search(const st_position* pos, int32_t P, int32_t S, int32_t depth, uint64_t seed,
                    const uint32_t* stream_ids, const float* pi_theta, const float* q_values, double alpha,
                    double beta,
                    const st_rules* rules, int32_t* n_moves, int16_t* actions, int32_t* tallies, double* q,
                    double* pi, int16_t* chosen, uint8_t* item_status, void* stream);

/*
 * Serving: test-time search requests with continuous batching (App. E: one
 * search per move; here the search is st_rollout's belief samples and
 * rollouts, with the rules' rollout policy).
 *
 * The server owns, from st_serve_create on: max_requests request slots on
 * the device (root position, root state, counters), sample_slots per-sample
 * records (sampled hidden types and outcome of each rollout), max_batches
 * streams, and a scheduler thread.  A submitted request waits in arrival
 * order until a request slot, K contiguous sample records and a stream are
 * free (admission by free device memory); every request admitted since the
 * previous launch goes into one batch (one 8-lane team per (request,
 * sample), at most a resident grid striding over the batch).  Batches run
 * concurrently, so a request arriving while others run starts at once
 * instead of at a batch boundary.  A request's result is exactly
 * st_rollout's tallies for the same position, K, depth, seed and stream id.
 */
typedef struct st_server st_server;

typedef struct st_serve_config {
    int32_t device;              /* CUDA device ordinal */
    int32_t max_requests;        /* request slots resident at once, 1..65536 */
    int32_t sample_slots;        /* per-sample records resident at once, 1..2^26 */
    int32_t max_batches;         /* batches in flight at once (streams), 1..64 */
    st_rules rules;
} st_serve_config;

typedef struct st_request {
    st_position pos;             /* HOST: root position (copied at submit) */
    int32_t K;                   /* belief samples, 0..sample_slots */
    int32_t depth;               /* rollout plies, >= 0 */
    uint64_t seed;               /* Philox key */
    uint32_t stream_id;          /* Philox counter word 0 (st_rollout's stream_ids[p]) */
} st_request;

typedef struct st_timing {
    uint64_t submit_ns;          /* steady-clock times of submit, admission, completion */
    uint64_t admit_ns;
    uint64_t done_ns;
} st_timing;

typedef struct st_serve_stats {
    int64_t submitted, admitted, completed, batches, max_batch_requests, queued, running;
} st_serve_stats;

st_status st_serve_create(const st_serve_config* cfg, st_server** out);
/* Queue a request (all HOST memory); returns a ticket at once, without
 * waiting for the scheduler.  ST_ERR_BUSY if 2^20 submissions wait to be
 * taken in. */
st_status st_serve_submit(st_server* srv, const st_request* req, uint64_t* ticket);
/* ST_OK with tallies[4] (HOST) and timing (HOST, may be NULL) once done, then
 * the ticket is released; ST_ERR_NOT_READY before; ST_ERR_BAD_POSITION if the
 * root failed validation (tallies zero); ST_ERR_INVALID for an unknown ticket. */
st_status st_serve_poll(st_server* srv, uint64_t ticket, int32_t* tallies, st_timing* timing);
/* As st_serve_poll, blocking up to timeout_ms; ST_ERR_TIMEOUT if not done. */
st_status st_serve_wait(st_server* srv, uint64_t ticket, int32_t timeout_ms, int32_t* tallies, st_timing* timing);
st_status st_serve_get_stats(st_server* srv, st_serve_stats* out);
/* Stops the scheduler, waits for launched batches, frees everything. */
st_status st_serve_destroy(st_server* srv);

#ifdef __cplusplus
}
#endif

#endif
