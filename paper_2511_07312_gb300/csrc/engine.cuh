// engine.cuh -- warp-cooperative Stratego engine for sm_103a.
//
// One warp owns one game at a time.  The game lives in a warp-private
// shared-memory record (SmemGame): the 288-byte per-game state that persists
// in HBM between launches, the board rebuilt from it (piece id per square),
// and the 1,264-byte legal-move mask of the player to move.  Lanes split the
// work of mask generation (one task per (movable piece, direction), compacted
// with __ballot_sync / __popc) and of setup, hashing and output; the scalar
// part of a ply (apply, battle, rule state) runs on lane 0.
//
// Rules follow App. A of arXiv 2511.07312 (Tab. pieces, Tab. chase), the
// two-square and chasing state machines of App. B.2-B.3, the k-move rule and
// cap of App. D.1 (Tab. game-hyper).  Where the paper is silent the same
// readings as the rest of this library apply: threats and evades are
// non-battle moves, evade takes precedence over threat, a chase position is
// the piece-id occupancy after one of the chaser's threats, and endings are
// checked flag / no legal move / k rule / cap, in that order.
//
// Chase positions are kept as 64-bit Zobrist-style hashes of (piece, square)
// pairs (splitmix64 finalizer over the pair index); a hash equality stands
// for board equality.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace stg {

constexpr int kPieces = 80;
constexpr int kSquares = 100;
constexpr uint8_t kEmpty = 0xFF;
constexpr uint8_t kLake = 0xFE;
constexpr uint8_t kNone = 0xFF;
constexpr int kMaskBytes = 1264;
constexpr int kMaskWordsAlloc = 320;   // 316 used by the output layout, 4 spare (kept zero)
constexpr int kPiCap = 128;            // chase positions per game (k <= 255 -> <= 128 threats)
constexpr int kRing = 256;             // moves of history per game

enum : int { kSpy = 0, kScout = 1, kMiner = 2, kMarshal = 9, kFlag = 10, kBomb = 11 };
enum : int { kClBattle = 0, kClQuiet = 1, kClThreat = 2, kClEvade = 3 };

constexpr uint32_t kTwoSquare = 1u, kChase = 2u, kAutoreset = 4u;

struct Rules {
    int k;          // battleless limit
    int cap;        // max plies
    uint32_t flags; // rule bits (+ autoreset for envs)
};

// Persistent per-game record in HBM (288 bytes, 16-byte aligned).
struct __align__(16) GameCore {
    uint8_t type[80];
    uint8_t sq[80];
    uint8_t flags[80];      // bit0 alive, bit1 revealed, bit2 moved, bit3 scout-known, bits4-6 cause
    int16_t ply;
    int16_t battleless;
    uint8_t last_battle;
    uint8_t chaser;
    uint8_t chase_plies;
    uint8_t n_pi;
    uint8_t ts_pid[2];
    uint8_t ts_len[2];
    uint8_t ts_sq[2][4];
    uint8_t terminated;     // ending code of a finished game kept without auto-reset
    uint8_t pad0;
    uint16_t n_legal;
    uint32_t episode;
    uint32_t pad1;
    uint64_t hash;          // XOR of zkey(pid, square) over alive pieces
    uint64_t pad2;
};
static_assert(sizeof(GameCore) == 288, "GameCore layout");

struct __align__(16) SmemGame {
    GameCore c;
    uint8_t board[112];
    uint32_t mask[kMaskWordsAlloc];
};
static_assert(sizeof(SmemGame) == 288 + 112 + 1280, "SmemGame layout");

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// ----------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11).
__device__ __forceinline__ uint4 philox(uint4 ctr, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t lo0 = ctr.x * 0xD2511F53u, hi0 = __umulhi(ctr.x, 0xD2511F53u);
        const uint32_t lo1 = ctr.z * 0xCD9E8D57u, hi1 = __umulhi(ctr.z, 0xCD9E8D57u);
        ctr = make_uint4(hi1 ^ ctr.y ^ k0, lo1, hi0 ^ ctr.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return ctr;
}

__device__ __forceinline__ uint32_t uniform_below(uint32_t r, uint32_t n) { return __umulhi(r, n); }

// ----------------------------------------------------------------- hashing
__device__ __forceinline__ uint64_t zkey(uint32_t pid, uint32_t square)
{
    uint64_t x = (uint64_t)(pid * 128u + square + 1u) * 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// ----------------------------------------------------------------- geometry
__device__ __forceinline__ bool is_lake(int s)
{
    const int r = s / 10, c = s - 10 * (s / 10);
    return (r == 4 || r == 5) && (c == 2 || c == 3 || c == 6 || c == 7);
}
__device__ __forceinline__ bool adjacent(int a, int b)
{
    const int ra = a / 10, ca = a - 10 * ra, rb = b / 10, cb = b - 10 * rb;
    return abs(ra - rb) + abs(ca - cb) == 1;
}
__device__ __forceinline__ int start_square(int pid) { return pid < 40 ? pid : pid + 20; }

// Sorted multiset of one side's 40 pieces (Tab. pieces counts, type-code order).
__device__ __forceinline__ uint8_t sorted_type(int k)
{
    // cumulative counts: Spy 1, Scout 8, Miner 5, Sergeant 4, Lieutenant 4,
    // Captain 4, Major 3, Colonel 2, General 1, Marshal 1, Flag 1, Bomb 6
    constexpr int ends[12] = {1, 9, 14, 18, 22, 26, 29, 31, 32, 33, 34, 40};
    int t = 0;
#pragma unroll
    for (int i = 0; i < 11; ++i) t += (k >= ends[i]);
    return (uint8_t)t;
}

__device__ __forceinline__ int nth_set_bit(uint32_t m, int n)
{
    int pos = 0, c;
    c = __popc(m & 0xFFFFu); if (n >= c) { n -= c; m >>= 16; pos += 16; }
    c = __popc(m & 0xFFu);   if (n >= c) { n -= c; m >>= 8;  pos += 8; }
    c = __popc(m & 0xFu);    if (n >= c) { n -= c; m >>= 4;  pos += 4; }
    c = __popc(m & 0x3u);    if (n >= c) { n -= c; m >>= 2;  pos += 2; }
    c = (int)(m & 1u);       if (n >= c) { pos += 1; }
    return pos;
}

// ----------------------------------------------------------------- state load/store
__device__ __forceinline__ void load_core(SmemGame* G, const GameCore* src)
{
    const int lane = lane_id();
    if (lane < 18) reinterpret_cast<uint4*>(&G->c)[lane] = reinterpret_cast<const uint4*>(src)[lane];
    __syncwarp();
}
__device__ __forceinline__ void store_core(const SmemGame* G, GameCore* dst)
{
    __syncwarp();
    const int lane = lane_id();
    if (lane < 18) reinterpret_cast<uint4*>(dst)[lane] = reinterpret_cast<const uint4*>(&G->c)[lane];
}

__device__ __forceinline__ void build_board(SmemGame* G)
{
    const int lane = lane_id();
    for (int s = lane; s < 112; s += 32) G->board[s] = (s < 100 && is_lake(s)) ? kLake : kEmpty;
    __syncwarp();
    for (int p = lane; p < kPieces; p += 32)
        if (G->c.flags[p] & 1) G->board[G->c.sq[p]] = (uint8_t)p;
    __syncwarp();
}

__device__ __forceinline__ uint64_t warp_xor64(uint64_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v ^= __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

__device__ __forceinline__ uint64_t board_hash(const SmemGame* G)
{
    const int lane = lane_id();
    uint64_t h = 0;
    for (int p = lane; p < kPieces; p += 32)
        if (G->c.flags[p] & 1) h ^= zkey(p, G->c.sq[p]);
    return warp_xor64(h);
}

// History: the action played i+1 plies ago, 0xFFFF if unknown.
__device__ __forceinline__ int hist_at(const SmemGame* G, const uint16_t* ring, int i)
{
    const int ply = G->c.ply;
    if (i >= ply || i >= kRing) return 0xFFFF;
    return ring[(ply - 1 - i) & (kRing - 1)];
}

// ----------------------------------------------------------------- rule context
struct PlyCtx {
    int prev_to;        // square the previous ply ended on (-1 none)
    int prev_nb;        // previous ply was not a battle
    int h1_from, h1_to; // the move played two plies ago (-1 none)
};

__device__ __forceinline__ PlyCtx make_ctx(const SmemGame* G, const uint16_t* ring)
{
    PlyCtx x;
    const int h0 = hist_at(G, ring, 0), h1 = hist_at(G, ring, 1);
    x.prev_to = h0 == 0xFFFF ? -1 : h0 % 100;
    x.prev_nb = !G->c.last_battle;
    x.h1_from = h1 == 0xFFFF ? -1 : h1 / 100;
    x.h1_to = h1 == 0xFFFF ? -1 : h1 % 100;
    return x;
}

__device__ __forceinline__ bool enemy_of(uint8_t o, int P) { return o < kPieces && (int)(o / 40) != P; }

__device__ __forceinline__ bool threat_square(const SmemGame* G, int q, int P)
{
    const int r = q / 10, c = q - 10 * r;
    bool t = false;
    if (r > 0) t |= enemy_of(G->board[q - 10], P);
    if (r < 9) t |= enemy_of(G->board[q + 10], P);
    if (c > 0) t |= enemy_of(G->board[q - 1], P);
    if (c < 9) t |= enemy_of(G->board[q + 1], P);
    return t;
}

__device__ __forceinline__ int classify(const SmemGame* G, const PlyCtx& x, int P, int from, int to)
{
    if (G->board[to] != kEmpty) return kClBattle;
    if (x.prev_to >= 0 && x.prev_nb && enemy_of(G->board[x.prev_to], P) && adjacent(from, x.prev_to) &&
        !adjacent(to, x.prev_to))
        return kClEvade;
    return threat_square(G, to, P) ? kClThreat : kClQuiet;
}

// Two-square rule: the 4th consecutive move of the same piece along one line
// is illegal if some square boundary lies inside all four moves' spans.
__device__ __forceinline__ bool two_square_blocks(const SmemGame* G, int P, int to)
{
    const uint8_t* p = G->c.ts_sq[P];
    const int s0 = p[0], s1 = p[1], s2 = p[2], s3 = p[3];
    const int r0 = s0 / 10, r1 = s1 / 10, r2 = s2 / 10, r3 = s3 / 10, r4 = to / 10;
    const int c0 = s0 - 10 * r0, c1 = s1 - 10 * r1, c2 = s2 - 10 * r2, c3 = s3 - 10 * r3, c4 = to - 10 * r4;
    const bool same_row = r0 == r1 && r0 == r2 && r0 == r3 && r0 == r4;
    const bool same_col = c0 == c1 && c0 == c2 && c0 == c3 && c0 == c4;
    if (!same_row && !same_col) return false;
    const int a0 = same_row ? c0 : r0, a1 = same_row ? c1 : r1, a2 = same_row ? c2 : r2;
    const int a3 = same_row ? c3 : r3, a4 = same_row ? c4 : r4;
    const int lo = max(max(min(a0, a1), min(a1, a2)), max(min(a2, a3), min(a3, a4)));
    const int hi = min(min(max(a0, a1), max(a1, a2)), min(max(a2, a3), max(a3, a4)));
    return lo < hi;
}

__device__ __forceinline__ bool chase_blocks(const SmemGame* G, const PlyCtx& x, const uint64_t* pi, int P,
                                             int pid, int from, int to)
{
    if (classify(G, x, P, from, to) != kClThreat) return false;
    if (from == x.h1_to && to == x.h1_from) return false;
    const uint64_t h = G->c.hash ^ zkey(pid, from) ^ zkey(pid, to);
    const int n = G->c.n_pi;
    for (int i = 0; i < n; ++i)
        if (pi[i] == h) return true;
    return false;
}

// ----------------------------------------------------------------- move generation
// Counts (and, if write_mask, records in G->mask) the moves of player P.
// physical: movement rules only (App. A "Piece details"); otherwise the
// two-square and chasing rules filter as rules.flags says.  Returns the
// warp-uniform count.
static __device__ __noinline__ int gen_moves(SmemGame* G, int P, uint32_t rule_flags, bool physical, bool write_mask,
                                      const uint16_t* ring, const uint64_t* pi)
{
    const int lane = lane_id();
    if (write_mask) {
        uint4* m4 = reinterpret_cast<uint4*>(G->mask);
        const uint4 z = make_uint4(0, 0, 0, 0);
        for (int i = lane; i < kMaskWordsAlloc / 4; i += 32) m4[i] = z;
    }
    const int base = P * 40;
    const uint8_t f0 = G->c.flags[base + lane], t0 = G->c.type[base + lane];
    const uint32_t b0 = __ballot_sync(0xFFFFFFFFu, (f0 & 1) && t0 < kFlag);
    bool ok1 = false;
    if (lane < 8) {
        const uint8_t f1 = G->c.flags[base + 32 + lane], t1 = G->c.type[base + 32 + lane];
        ok1 = (f1 & 1) && t1 < kFlag;
    }
    const uint32_t b1 = __ballot_sync(0xFFFFFFFFu, ok1);
    const int n0 = __popc(b0), npieces = n0 + __popc(b1);

    const bool ts_on = !physical && (rule_flags & kTwoSquare) && G->c.ts_pid[P] != kNone && G->c.ts_len[P] == 4;
    const int ts_pid = G->c.ts_pid[P];
    const bool chase_on = !physical && (rule_flags & kChase) && G->c.chaser == P && G->c.n_pi > 0;
    PlyCtx x;
    if (chase_on) x = make_ctx(G, ring);
    __syncwarp();

    int cnt = 0;
    const int ntasks = npieces * 4;
    for (int task = lane; task < ntasks; task += 32) {
        const int k = task >> 2, dir = task & 3;
        const int j = k < n0 ? nth_set_bit(b0, k) : 32 + nth_set_bit(b1, k - n0);
        const int pid = base + j;
        const int s = G->c.sq[pid];
        const int r = s / 10, c = s - 10 * r;
        const int dr = (dir == 0) - (dir == 1), dc = (dir == 2) - (dir == 3);
        const int maxd = G->c.type[pid] == kScout ? 9 : 1;
        for (int d = 1; d <= maxd; ++d) {
            const int rr = r + dr * d, cc = c + dc * d;
            if ((unsigned)rr > 9u || (unsigned)cc > 9u) break;
            const int q = rr * 10 + cc;
            const uint8_t occ = G->board[q];
            if (occ == kLake) break;
            const bool enemy = occ != kEmpty;
            if (enemy && (int)(occ / 40) == P) break;
            bool legal = true;
            if (ts_on && pid == ts_pid) legal = !two_square_blocks(G, P, q);
            if (legal && chase_on && !enemy) legal = !chase_blocks(G, x, pi, P, pid, s, q);
            if (legal) {
                ++cnt;
                if (write_mask) {
                    const int a = s * 100 + q;
                    atomicOr(&G->mask[a >> 5], 1u << (a & 31));
                }
            }
            if (enemy) break;
        }
    }
    const int n = __reduce_add_sync(0xFFFFFFFFu, cnt);
    __syncwarp();
    return n;
}

// The idx-th set bit (ascending) of G->mask; warp-uniform result.
__device__ __forceinline__ int select_action(const SmemGame* G, uint32_t idx)
{
    const int lane = lane_id();
    uint32_t w[10];
    int cnt = 0;
#pragma unroll
    for (int k = 0; k < 10; ++k) {
        w[k] = G->mask[lane * 10 + k];
        cnt += __popc(w[k]);
    }
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += v;
    }
    const int excl = incl - cnt;
    const uint32_t own = __ballot_sync(0xFFFFFFFFu, (int)idx >= excl && (int)idx < incl);
    int a = -1;
    if (own & (1u << lane)) {
        int local = (int)idx - excl;
#pragma unroll
        for (int k = 0; k < 10; ++k) {
            const int ck = __popc(w[k]);
            if (a < 0 && local < ck) a = (lane * 10 + k) * 32 + nth_set_bit(w[k], local);
            if (a < 0) local -= ck;
        }
    }
    const int src = own ? __ffs(own) - 1 : 0;
    return __shfl_sync(0xFFFFFFFFu, a, src);
}

__device__ __forceinline__ bool mask_has(const SmemGame* G, int a)
{
    return a >= 0 && a < 10000 && ((G->mask[a >> 5] >> (a & 31)) & 1u);
}

// Is the flag of `side` captured?
__device__ __forceinline__ bool flag_dead(const SmemGame* G, int side)
{
    const int lane = lane_id();
    bool d = false;
    for (int k = lane; k < 40; k += 32) {
        const int p = side * 40 + k;
        d |= G->c.type[p] == kFlag && !(G->c.flags[p] & 1);
    }
    return __any_sync(0xFFFFFFFFu, d);
}

// ----------------------------------------------------------------- apply
// Plays action a for the player to move.  ring/pi: this game's history ring
// and chase-position store.  Returns whether the move was a battle.
static __device__ __noinline__ void apply_move(SmemGame* G, int a, uint16_t* ring, uint64_t* pi)
{
    const int lane = lane_id();
    if (a < 0 || a >= 10000) return;   // callers pass mask members only; never index outside the board
    const PlyCtx x = make_ctx(G, ring);
    __syncwarp();
    if (lane == 0) {
        GameCore& c = G->c;
        const int P = c.ply & 1;
        const int from = a / 100, to = a - 100 * (a / 100);
        const int X = G->board[from];
        const int cls = classify(G, x, P, from, to);
        const int dist = abs(from - to) >= 10 ? abs(from - to) / 10 : abs(from - to);
        uint8_t fx = c.flags[X];
        if (dist > 1) fx |= 8;
        fx |= 4;
        const bool battle = G->board[to] != kEmpty;
        uint64_t h = c.hash ^ zkey(X, from);
        int D = -1;
        bool d_died = false, x_alive = true;
        G->board[from] = kEmpty;
        if (!battle) {
            G->board[to] = (uint8_t)X;
            c.sq[X] = (uint8_t)to;
            h ^= zkey(X, to);
        } else {
            D = G->board[to];
            uint8_t fd = c.flags[D];
            const bool d_rev = fd & 2;
            const int ta = c.type[X], td = c.type[D];
            // Tab. pieces: Flag loses to any attacker; Bomb beats all but the
            // Miner; the attacking Spy beats the Marshal; otherwise by rank.
            int out;
            if (td == kFlag) out = 1;
            else if (td == kBomb) out = ta == kMiner ? 1 : 2;
            else if (ta == kSpy && td == kMarshal) out = 1;
            else out = ta > td ? 1 : (ta < td ? 2 : 3);
            fx |= 2;
            fd |= 2;
            if (out == 1) {
                fd = (uint8_t)((fd & 0x0E) | ((d_rev ? 4 : 6) << 4));
                d_died = true;
                G->board[to] = (uint8_t)X;
                c.sq[X] = (uint8_t)to;
                h ^= zkey(D, to) ^ zkey(X, to);
            } else if (out == 2) {
                fx = (uint8_t)((fx & 0x0E) | ((d_rev ? 1 : 3) << 4));
                c.sq[X] = (uint8_t)to;
                x_alive = false;
            } else {
                fx = (uint8_t)((fx & 0x0E) | ((d_rev ? 2 : 3) << 4));
                fd = (uint8_t)((fd & 0x0E) | ((d_rev ? 5 : 6) << 4));
                c.sq[X] = (uint8_t)to;
                d_died = true;
                x_alive = false;
                G->board[to] = kEmpty;
                h ^= zkey(D, to);
            }
            c.flags[D] = fd;
        }
        c.flags[X] = fx;
        c.hash = h;
        const int ply_before = c.ply;
        c.battleless = battle ? 0 : (int16_t)(c.battleless + 1);
        c.last_battle = battle ? 1 : 0;
        c.ply = (int16_t)(c.ply + 1);
        // two-square state
        if (!x_alive) {
            c.ts_pid[P] = kNone; c.ts_len[P] = 0;
            c.ts_sq[P][0] = c.ts_sq[P][1] = c.ts_sq[P][2] = c.ts_sq[P][3] = kNone;
        } else if (c.ts_pid[P] == X && c.ts_len[P] >= 2) {
            if (c.ts_len[P] == 4) {
                c.ts_sq[P][0] = c.ts_sq[P][1]; c.ts_sq[P][1] = c.ts_sq[P][2];
                c.ts_sq[P][2] = c.ts_sq[P][3]; c.ts_sq[P][3] = (uint8_t)to;
            } else {
                c.ts_sq[P][c.ts_len[P]] = (uint8_t)to;
                c.ts_len[P] += 1;
            }
        } else {
            c.ts_pid[P] = (uint8_t)X; c.ts_len[P] = 2;
            c.ts_sq[P][0] = (uint8_t)from; c.ts_sq[P][1] = (uint8_t)to;
            c.ts_sq[P][2] = c.ts_sq[P][3] = kNone;
        }
        if (d_died && c.ts_pid[1 - P] == D) {
            c.ts_pid[1 - P] = kNone; c.ts_len[1 - P] = 0;
            c.ts_sq[1 - P][0] = c.ts_sq[1 - P][1] = c.ts_sq[1 - P][2] = c.ts_sq[1 - P][3] = kNone;
        }
        // chase state
        if (cls == kClThreat) {
            if (c.chaser != P) { c.chaser = (uint8_t)P; c.n_pi = 0; c.chase_plies = 0; }
            if (c.n_pi < kPiCap) { pi[c.n_pi] = h; c.n_pi += 1; }
            c.chase_plies += 1;
        } else if (cls == kClEvade && c.chaser == 1 - P) {
            c.chase_plies += 1;
        } else {
            c.chaser = kNone; c.n_pi = 0; c.chase_plies = 0;
        }
        ring[ply_before & (kRing - 1)] = (uint16_t)a;
    }
    __syncwarp();
}

// ----------------------------------------------------------------- new game
// setup: custom types per piece id, or nullptr for the Philox setup of
// (slot, episode).
static __device__ __noinline__ void reset_game(SmemGame* G, uint32_t k0, uint32_t k1, uint32_t slot, uint32_t episode,
                                        const uint8_t* setup)
{
    const int lane = lane_id();
    for (int p = lane; p < kPieces; p += 32) {
        G->c.type[p] = setup ? setup[p] : sorted_type(p % 40);
        G->c.sq[p] = (uint8_t)start_square(p);
        G->c.flags[p] = 1;
    }
    __syncwarp();
    if (!setup && lane < 2) {
        uint8_t* arr = G->c.type + 40 * lane;
        uint4 w = make_uint4(0, 0, 0, 0);
        for (int i = 39; i >= 1; --i) {
            const int d = 39 - i;
            if ((d & 3) == 0)
                w = philox(make_uint4(slot, episode, 0u, (1u << 24) | ((uint32_t)lane << 8) | (uint32_t)(d >> 2)),
                           k0, k1);
            const uint32_t r = (d & 3) == 0 ? w.x : (d & 3) == 1 ? w.y : (d & 3) == 2 ? w.z : w.w;
            const uint32_t j = uniform_below(r, (uint32_t)(i + 1));
            const uint8_t t = arr[i];
            arr[i] = arr[j];
            arr[j] = t;
        }
    }
    if (lane == 0) {
        GameCore& c = G->c;
        c.ply = 0; c.battleless = 0; c.last_battle = 0;
        c.chaser = kNone; c.chase_plies = 0; c.n_pi = 0;
        c.ts_pid[0] = c.ts_pid[1] = kNone; c.ts_len[0] = c.ts_len[1] = 0;
        for (int i = 0; i < 4; ++i) c.ts_sq[0][i] = c.ts_sq[1][i] = kNone;
        c.terminated = 0; c.episode = episode; c.n_legal = 0;
    }
    __syncwarp();
    const uint64_t h = board_hash(G);
    if (lane == 0) G->c.hash = h;
    build_board(G);
}

// ----------------------------------------------------------------- one ply of the env loop
struct PlyResult {
    int action;
    int code;
    int winner;
    int ply_idx;
};

// Ending after the ply just played (App. A "Game Summary", App. D.1); also
// leaves the mask of the player to move in G->mask and its count in n.
__device__ __forceinline__ void check_end(SmemGame* G, const Rules& R, const uint16_t* ring, const uint64_t* pi,
                                          int& code, int& winner, int& n)
{
    const int Q = G->c.ply & 1, P = 1 - Q;
    code = 0;
    winner = -1;
    n = 0;
    if (flag_dead(G, Q)) { code = 1; winner = P; return; }
    n = gen_moves(G, Q, R.flags, false, true, ring, pi);
    if (n == 0) {
        const int phys = gen_moves(G, P, R.flags, true, false, ring, pi);
        code = phys == 0 ? 3 : 2;
        winner = phys == 0 ? -1 : P;
        return;
    }
    if (G->c.battleless >= R.k) { code = 4; return; }
    if (G->c.ply >= R.cap) { code = 5; return; }
}

// The acting player of a fresh position has no legal move (n_legal == 0).
__device__ __forceinline__ void start_end(SmemGame* G, const Rules& R, const uint16_t* ring, const uint64_t* pi,
                                          int& code, int& winner)
{
    const int P = G->c.ply & 1;
    const int phys = gen_moves(G, 1 - P, R.flags, true, false, ring, pi);
    code = phys == 0 ? 3 : 2;
    winner = phys == 0 ? -1 : 1 - P;
}

__device__ __forceinline__ void zero_mask(SmemGame* G)
{
    uint4* m4 = reinterpret_cast<uint4*>(G->mask);
    for (int i = lane_id(); i < kMaskWordsAlloc / 4; i += 32) m4[i] = make_uint4(0, 0, 0, 0);
    __syncwarp();
}

}  // namespace stg
