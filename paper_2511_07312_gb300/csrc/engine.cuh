// engine.cuh -- team-cooperative Stratego engine for sm_103a.
//
// A team of L lanes (L = 32, 16, 8 or 4: 1, 2, 4 or 8 games per warp) owns
// one game at a time.  The game lives in a team-private shared-memory record
// (SmemGame, 1,168 bytes): the 288-byte per-game state that persists in HBM
// between launches, the board (piece id per square), 128-bit square sets
// kept up to date ply by ply (own pieces, movable non-Scouts and Scouts per
// player), occupancy per column, and the moves of the player to move as a
// count and a descriptor per from-square.  The 1,264-byte legal mask is an
// output only: the move generator writes it straight into the caller's row
// in global memory (no shared-memory copy of it is kept).
//
// Move generation: non-Scout moves of the whole board come from four shifted
// square sets; lane j of the team records those of its segment of 25, 13, 7
// or 4 from-squares (L = 4, 8, 16, 32), each from-square's (at most four)
// destinations as one window of at most 21 mask bits (plain stores: two
// windows never share a 32-bit word).  Each Scout takes one lane (two on
// 4-lane teams); its slides come from the row and column occupancy with
// find-first-set, and its mask bits are ORed in word by word.  A move is
// chosen from the per-square counts (which square) and the square's
// descriptor (which destination), not from the mask.  The scalar part of a
// ply (apply, battle, rule state) runs on the team's first lane; all
// collectives are team-masked, so the teams of a warp run in lockstep when
// their games take the same path and serialize harmlessly when they do not.
// A team's lanes reach every collective together: where lanes read a value
// that a later phase rewrites (the ending of a ply before a restart, the
// records before an illegal action's re-generation) a team barrier separates
// the reads from the writes.
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
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace stg {

constexpr int kPieces = 80;
constexpr int kSquares = 100;
constexpr uint8_t kEmpty = 0xFF;
constexpr uint8_t kLake = 0xFE;
constexpr uint8_t kNone = 0xFF;
constexpr int kMaskBytes = 1264;
constexpr int kMaskWordsAlloc = 316;   // the output layout: 1,264 bytes
constexpr int kSegMax = 25;            // from-square segments (one per lane; 25 of 4 squares for 32 lanes)
constexpr int kCntBytes = 128;         // per-square move counts: 100 squares padded to 128 bytes
// Move descriptor of a from-square (SmemGame::desc, 16 bits): a non-Scout's
// legal moves as kDescStep | bits 0-3 (to s-10, s-1, s+1, s+10); a Scout's as
// south | west << 4 | east << 8 | north << 12 (squares slid in each
// direction, the capture included: at most 9 each, so neither marker is a
// Scout's); a Scout some of whose moves a rule forbids as kDescFiltered (its
// moves are rebuilt on demand).
constexpr uint16_t kDescStep = 0xFFF0u, kDescFiltered = 0xEEEEu;
constexpr int kPiCap = 128;            // chase positions per game (k <= 255 -> <= 128 threats)
constexpr int kPiWords = 2 * kPiCap;   // each: hash of the chaser's pieces, hash of the chased side's pieces
constexpr int kRing = 256;             // moves of history per game
constexpr uint32_t kLakeRow = 0xCCu;   // columns 2,3,6,7 of rows 4 and 5
constexpr uint32_t kLakeCol = 0x30u;   // rows 4,5 of columns 2,3,6,7

enum : int { kSpy = 0, kScout = 1, kMiner = 2, kMarshal = 9, kFlag = 10, kBomb = 11 };
enum : int { kClBattle = 0, kClQuiet = 1, kClThreat = 2, kClEvade = 3 };

constexpr uint32_t kTwoSquare = 1u, kChase = 2u, kAutoreset = 4u, kMagnet = 0x100u;
// How a game began (env history): a new game (Philox setup, pool or pin), a
// reset to given setups, an imported snapshot.
enum : uint8_t { kFreshNew = 1, kFreshSetup = 2, kFreshImport = 3 };

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
    uint8_t fresh;          // env history: this state began a game (kFresh*), 0 once a step is recorded
    uint16_t n_legal;
    uint32_t episode;
    uint16_t hrow;          // env history: ring row of the next step
    uint16_t hcur;          // env history: the fresh mark of the ply being played
    uint64_t hash_side[2];  // per side: XOR of zkey(pid, square) over its alive pieces
};
static_assert(sizeof(GameCore) == 288, "GameCore layout");

// Square sets: bit s of a 128-bit set is square s; word 0 holds squares
// 0-63, word 1 squares 64-99.
struct __align__(16) SmemGame {
    GameCore c;
    uint8_t board[112];
    uint64_t bocc[2][2];      // pieces of player p
    uint64_t bmov[2][2];      // movable non-Scouts of player p
    uint64_t bsco[2][2];      // Scouts of player p
    uint16_t colocc[10];      // all pieces in column c (bit = row)
    uint16_t h0, h1;          // actions played 1 and 2 plies ago (0xFFFF none)
    uint8_t flag_pid[2];
    uint8_t scout_pid[2][8];  // the Scouts of each side in piece-id order (kNone after the last)
    uint8_t gen_chase;        // the last generation filtered all moves by the chasing rule
    uint8_t pad[5];
    uint64_t pi_theirs[4];    // chased-side hash of chase positions n_pi-4 .. n_pi-1 (slot i & 3)
    uint64_t pi_mine[4];      // the chaser's hash of the same positions
    uint32_t stat[8];         // counters of the current launch (kept by the env's step loop)
    uint8_t sq_cnt[kCntBytes];// legal moves per from-square of the player to move (zero past square 99)
    // -- the descriptors come last: code that records moves as mask rows
    //    (gen_moves<L, true>, the persistent step) never touches them and
    //    keeps its records kRowsGameBytes apart
    uint16_t desc[kSquares];  // move descriptor per from-square (valid where sq_cnt > 0, see kDescStep)
    uint8_t pad2[8];
};
static_assert(sizeof(SmemGame) == 288 + 112 + 96 + 20 + 4 + 2 + 16 + 6 + 64 + 32 + kCntBytes + 2 * kSquares + 8,
              "SmemGame layout");
static_assert(offsetof(SmemGame, sq_cnt) % 16 == 0, "per-square counts are read as 16-byte words");
// A game record whose moves are recorded as mask rows (row mode, the
// persistent step) has no descriptors: its kRowsGameBytes are followed
// directly by the 1,264-byte mask of the player to move (rows_of), so that
// the per-square counts and the mask are one run of 16-byte words.
constexpr int kRowsGameBytes = (int)offsetof(SmemGame, desc);
constexpr int kRowsRecordBytes = kRowsGameBytes + kMaskBytes;
static_assert(kRowsGameBytes % 16 == 0 && kRowsGameBytes == (int)offsetof(SmemGame, sq_cnt) + kCntBytes,
              "row-mode records: counts then mask, 16-byte aligned");
__device__ __forceinline__ uint32_t* rows_of(SmemGame* G)
{
    return reinterpret_cast<uint32_t*>(reinterpret_cast<unsigned char*>(G) + kRowsGameBytes);
}
__device__ __forceinline__ const uint32_t* rows_of(const SmemGame* G)
{
    return reinterpret_cast<const uint32_t*>(reinterpret_cast<const unsigned char*>(G) + kRowsGameBytes);
}
static_assert(sizeof(SmemGame) % 16 == 0, "SmemGame alignment");
constexpr int kGameHead = 288 + 112;   // core + board: the part copied from a root

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// ----------------------------------------------------------------- teams
template <int L>
struct Team {
    static_assert(L == 32 || L == 16 || L == 8 || L == 4, "teams of 4, 8, 16 or 32 lanes");
    int tl;          // lane within the team
    int base;        // first warp lane of the team
    unsigned mask;   // warp lanes of the team
    __device__ __forceinline__ Team()
    {
        const int lane = threadIdx.x & 31;
        tl = lane & (L - 1);
        base = lane - tl;
        mask = L == 32 ? 0xFFFFFFFFu : (((1u << L) - 1u) << base);
    }
    __device__ __forceinline__ void sync() const { __syncwarp(mask); }
    __device__ __forceinline__ uint32_t ballot(bool p) const { return __ballot_sync(mask, p) >> base; }
    __device__ __forceinline__ bool any(bool p) const { return __any_sync(mask, p); }
    __device__ __forceinline__ int shfl(int v, int src) const { return __shfl_sync(mask, v, src, L); }
    __device__ __forceinline__ uint32_t shfl_up(uint32_t v, int d) const { return __shfl_up_sync(mask, v, d, L); }
    __device__ __forceinline__ uint32_t shfl_down(uint32_t v, int d) const { return __shfl_down_sync(mask, v, d, L); }
    __device__ __forceinline__ int sum(int v) const { return (int)__reduce_add_sync(mask, (unsigned)v); }
    __device__ __forceinline__ uint64_t xor64(uint64_t v) const
    {
#pragma unroll
        for (int o = L / 2; o > 0; o >>= 1) v ^= __shfl_xor_sync(mask, v, o, L);
        return v;
    }
    __device__ __forceinline__ bool leader() const { return tl == 0; }
};

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

// The n-th set bit (ascending) of a 64-bit word.
__device__ __forceinline__ int nth_set_bit64(uint64_t x, int n)
{
    const uint32_t lo = (uint32_t)x;
    const int cl = __popc(lo);
    return n < cl ? nth_set_bit(lo, n) : 32 + nth_set_bit((uint32_t)(x >> 32), n - cl);
}

__device__ __forceinline__ bool enemy_of(uint8_t o, int P) { return o < kPieces && (int)(o / 40) != P; }

// ----------------------------------------------------------------- state load/store
template <int L>
__device__ __forceinline__ void load_core(SmemGame* G, const GameCore* src, const Team<L>& T)
{
    for (int i = T.tl; i < 18; i += L) reinterpret_cast<uint4*>(&G->c)[i] = reinterpret_cast<const uint4*>(src)[i];
    T.sync();
}
template <int L>
__device__ __forceinline__ void store_core(const SmemGame* G, GameCore* dst, const Team<L>& T)
{
    T.sync();
    for (int i = T.tl; i < 18; i += L) reinterpret_cast<uint4*>(dst)[i] = reinterpret_cast<const uint4*>(&G->c)[i];
}

// History: the action played i+1 plies ago, 0xFFFF if unknown.
__device__ __forceinline__ int hist_at(const SmemGame* G, const uint16_t* ring, int i)
{
    const int ply = G->c.ply;
    if (i >= ply || i >= kRing) return 0xFFFF;
    return ring[(ply - 1 - i) & (kRing - 1)];
}

__device__ __forceinline__ void bb_set(uint64_t* b, int s) { b[s >> 6] |= 1ull << (s & 63); }
__device__ __forceinline__ void bb_clr(uint64_t* b, int s) { b[s >> 6] &= ~(1ull << (s & 63)); }

// Everything derived from the core and the board: square sets per player,
// column occupancy, flag ids, Scout lists, the last two moves, the cached
// hashes of the newest four chase positions (from the store pi).
// Needs G->board.  Each side has at most 8 Scouts (Tab. pieces; setups, imported
// positions and belief samples keep the piece counts).
template <int L>
__device__ __noinline__ void derive_state(SmemGame* G, const uint16_t* ring, const uint64_t* pi, Team<L>)
{
    // out-of-line engine functions rebuild the team from the lane id rather
    // than reading the caller's copy through memory
    const Team<L> T;
    uint64_t* sets = &G->bocc[0][0];   // bocc, bmov, bsco: 12 words
    for (int i = T.tl; i < 12; i += L) sets[i] = 0;
    T.sync();
    for (int p = T.tl; p < kPieces; p += L) {
        const int t = G->c.type[p], side = p / 40;
        if (t == kFlag) G->flag_pid[side] = (uint8_t)p;
        if (!(G->c.flags[p] & 1)) continue;
        const int s = G->c.sq[p];
        const unsigned long long b = 1ull << (s & 63);
        atomicOr(reinterpret_cast<unsigned long long*>(&G->bocc[side][s >> 6]), b);
        if (t == kScout) atomicOr(reinterpret_cast<unsigned long long*>(&G->bsco[side][s >> 6]), b);
        else if (t < kFlag) atomicOr(reinterpret_cast<unsigned long long*>(&G->bmov[side][s >> 6]), b);
    }
    for (int side = 0; side < 2; ++side) {
        int n = 0;
        for (int k0 = 0; k0 < 40; k0 += L) {
            const int k = k0 + T.tl;
            const bool is = k < 40 && G->c.type[40 * side + k] == kScout;
            const uint32_t b = T.ballot(is);
            const int rank = n + __popc(b & ((1u << T.tl) - 1u));
            if (is && rank < 8) G->scout_pid[side][rank] = (uint8_t)(40 * side + k);
            n += __popc(b);
        }
        for (int i = n + T.tl; i < 8; i += L) G->scout_pid[side][i] = kNone;
    }
    for (int c = T.tl; c < 10; c += L) {
        uint32_t col = 0;
        for (int r = 0; r < 10; ++r)
            if (G->board[10 * r + c] < kPieces) col |= 1u << r;
        G->colocc[c] = (uint16_t)col;
    }
    const int npi = G->c.n_pi;
    for (int i = max(npi - 4, 0) + T.tl; i < npi; i += L) {
        G->pi_mine[i & 3] = pi[2 * i];
        G->pi_theirs[i & 3] = pi[2 * i + 1];
    }
    if (T.leader()) {
        G->h0 = (uint16_t)hist_at(G, ring, 0);
        G->h1 = (uint16_t)hist_at(G, ring, 1);
    }
    T.sync();
}

template <int L>
__device__ __forceinline__ void build_board(SmemGame* G, const Team<L>& T)
{
    for (int s = T.tl; s < 112; s += L) G->board[s] = (s < 100 && is_lake(s)) ? kLake : kEmpty;
    T.sync();
    for (int p = T.tl; p < kPieces; p += L)
        if (G->c.flags[p] & 1) G->board[G->c.sq[p]] = (uint8_t)p;
    T.sync();
}

// Hash of the alive pieces of `side` (pieces 40*side .. 40*side+39).
template <int L>
__device__ __forceinline__ uint64_t side_hash(const SmemGame* G, const Team<L>& T, int side)
{
    uint64_t h = 0;
    for (int k = T.tl; k < 40; k += L) {
        const int p = 40 * side + k;
        if (G->c.flags[p] & 1) h ^= zkey(p, G->c.sq[p]);
    }
    return T.xor64(h);
}

// ----------------------------------------------------------------- rule context
struct PlyCtx {
    int prev_to;        // square the previous ply ended on (-1 none)
    int prev_nb;        // previous ply was not a battle
    int h1_from, h1_to; // the move played two plies ago (-1 none)
};

__device__ __forceinline__ PlyCtx make_ctx(const SmemGame* G)
{
    PlyCtx x;
    const int h0 = G->h0, h1 = G->h1;
    x.prev_to = h0 == 0xFFFF ? -1 : h0 % 100;
    x.prev_nb = !G->c.last_battle;
    x.h1_from = h1 == 0xFFFF ? -1 : h1 / 100;
    x.h1_to = h1 == 0xFFFF ? -1 : h1 % 100;
    return x;
}

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

// Would P's move of `pid` recreate a position reached after one of P's
// threats in the current chase?  Chase positions are stored as (hash of the
// chaser's pieces, hash of the chased side's pieces).
__device__ __forceinline__ bool chase_blocks(const SmemGame* G, const PlyCtx& x, const uint64_t* pi, int P,
                                             int pid, int from, int to)
{
    if (classify(G, x, P, from, to) != kClThreat) return false;
    if (from == x.h1_to && to == x.h1_from) return false;
    const uint64_t mine = G->c.hash_side[P] ^ zkey(pid, from) ^ zkey(pid, to);
    const uint64_t theirs = G->c.hash_side[1 - P];
    const int n = min((int)G->c.n_pi, kPiCap);
    // the newest four positions from shared memory, older ones from the store
    for (int i = max(n - 4, 0); i < n; ++i)
        if (G->pi_theirs[i & 3] == theirs && G->pi_mine[i & 3] == mine) return true;
    for (int i = 0; i < n - 4; ++i)
        if (pi[2 * i + 1] == theirs && pi[2 * i] == mine) return true;
    return false;
}

// Can any of P's moves be chase-blocked?  A move of P changes only P's
// pieces, so a stored chase position can be recreated only if the chased
// side's pieces stand exactly where they stood then.  The newest four
// positions are checked in shared memory, older ones in the store.
// Team-uniform.
template <int L>
__device__ __forceinline__ bool chase_live(const SmemGame* G, const Team<L>& T, const uint64_t* pi, int P)
{
    const uint64_t theirs = G->c.hash_side[1 - P];
    const int n = min((int)G->c.n_pi, kPiCap);
    bool hit = T.tl < 4 && T.tl < n && G->pi_theirs[T.tl] == theirs;
    for (int i = T.tl; i < n - 4; i += L) hit |= pi[2 * i + 1] == theirs;
    return T.any(hit);
}

// 128-bit sets over to-squares, kept in registers as two 64-bit halves.
struct Set128 {
    uint64_t lo, hi;
};
__device__ __forceinline__ uint64_t lowbits64(int n) { return n <= 0 ? 0ull : (n >= 64 ? ~0ull : ((1ull << n) - 1ull)); }
// bits [a, a+n) (0 <= a, a+n <= 128)
__device__ __forceinline__ Set128 range128(int a, int n)
{
    Set128 r;
    const int b = a + n;
    r.lo = lowbits64(min(b, 64)) & ~lowbits64(min(a, 64));
    r.hi = lowbits64(max(b - 64, 0)) & ~lowbits64(max(a - 64, 0));
    return r;
}
__device__ __forceinline__ Set128 shl128(Set128 v, int s)   // 0 <= s < 128
{
    Set128 r;
    if (s == 0) return v;
    if (s >= 64) { r.hi = v.lo << (s - 64); r.lo = 0; return r; }
    r.hi = (v.hi << s) | (v.lo >> (64 - s));
    r.lo = v.lo << s;
    return r;
}
__device__ __forceinline__ Set128 or128(Set128 a, Set128 b) { return Set128{a.lo | b.lo, a.hi | b.hi}; }
__device__ __forceinline__ Set128 bit128(int i)
{
    return i < 64 ? Set128{1ull << i, 0ull} : Set128{0ull, 1ull << (i - 64)};
}
__device__ __forceinline__ int popc128(Set128 v) { return __popcll(v.lo) + __popcll(v.hi); }

// Squares c + 10k for k in [k0, k1] (column c, rows k0..k1).
__device__ __forceinline__ Set128 column128(int c, int k0, int k1)
{
    // bits 0, 10, 20, ..., 90
    const Set128 every10{0x1004010040100401ull, 0x0000000004010040ull};
    if (k1 < k0) return Set128{0, 0};
    // keep rows k0..k1 of the every-tenth pattern, then move to column c
    Set128 p = every10;
    const Set128 keep = range128(10 * k0, 10 * (k1 - k0) + 1);
    p.lo &= keep.lo;
    p.hi &= keep.hi;
    return shl128(p, c);
}

// Drops the destinations (128-bit set over to-squares) of the piece on
// `from` that the two-square or chasing rule forbids.
__device__ __forceinline__ Set128 filter_dests(const SmemGame* G, int P, int from, bool ts_here, bool chase_on,
                                               const PlyCtx& x, const uint64_t* pi, Set128 d)
{
    const int pid = G->board[from];
    for (int half = 0; half < 2; ++half) {
        uint64_t m = half ? d.hi : d.lo;
        while (m) {
            const int b = __ffsll(m) - 1;
            m &= m - 1;
            const int to = 64 * half + b;
            bool bad = ts_here && two_square_blocks(G, P, to);
            if (!bad && chase_on && G->board[to] == kEmpty) bad = chase_blocks(G, x, pi, P, pid, from, to);
            if (bad) {
                if (half) d.hi &= ~(1ull << b); else d.lo &= ~(1ull << b);
            }
        }
    }
    return d;
}

// OR bits 0..127 of d into the mask at bit offset base (bit i of d is mask
// bit base + i); only words that receive a set bit are touched.
__device__ __forceinline__ void or_bits(uint32_t* mask, int base, Set128 d)
{
    const int w0 = base >> 5, sh = base & 31;
    const uint32_t w[4] = {(uint32_t)d.lo, (uint32_t)(d.lo >> 32), (uint32_t)d.hi, (uint32_t)(d.hi >> 32)};
    uint32_t prev = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint32_t v = sh ? (w[i] << sh) | prev : w[i];
        prev = sh ? (w[i] >> (32 - sh)) : 0u;
        if (v) atomicOr(&mask[w0 + i], v);
    }
    if (prev) atomicOr(&mask[w0 + 4], prev);
}

// Bits a..b of a 32-bit word (clipped to 0..31; none if a > b after clipping).
__device__ __forceinline__ uint32_t range32(int a, int b)
{
    a = max(a, 0);
    b = min(b, 31);
    return a > b ? 0u : ((2u << b) - (1u << a));
}
// Square q (0..127) of a 128-bit set.
__device__ __forceinline__ bool test128(Set128 x, int q)
{
    return ((q < 64 ? x.lo >> q : x.hi >> (q - 64)) & 1ull) != 0;
}

// OR a 128-bit set over to-squares into the mask row of from-square s.
__device__ __forceinline__ void or_row(uint32_t* mask, int s, Set128 d) { or_bits(mask, 100 * s, d); }

// ----------------------------------------------------------------- square sets
constexpr uint64_t col_bits(int c, int half)
{
    uint64_t v = 0;
    for (int r = 0; r < 10; ++r) {
        const int s = 10 * r + c;
        if ((s >> 6) == half) v |= 1ull << (s & 63);
    }
    return v;
}
constexpr uint64_t kLakesLo = (1ull << 42) | (1ull << 43) | (1ull << 46) | (1ull << 47) | (1ull << 52) |
                              (1ull << 53) | (1ull << 56) | (1ull << 57);   // the lakes are squares < 64
constexpr uint64_t kValidHi = (1ull << 36) - 1ull;                         // squares 64-99
constexpr uint64_t kCol0Lo = col_bits(0, 0), kCol0Hi = col_bits(0, 1);
constexpr uint64_t kCol9Lo = col_bits(9, 0), kCol9Hi = col_bits(9, 1);

__device__ __forceinline__ Set128 ld128(const uint64_t* p) { return Set128{p[0], p[1]}; }
__device__ __forceinline__ Set128 and128(Set128 a, Set128 b) { return Set128{a.lo & b.lo, a.hi & b.hi}; }
// square s+k of the result is square s of the input (k = 1, 10) and back
__device__ __forceinline__ Set128 up1(Set128 a) { return Set128{a.lo << 1, (a.hi << 1) | (a.lo >> 63)}; }
__device__ __forceinline__ Set128 dn1(Set128 a) { return Set128{(a.lo >> 1) | (a.hi << 63), a.hi >> 1}; }
__device__ __forceinline__ Set128 up10(Set128 a) { return Set128{a.lo << 10, (a.hi << 10) | (a.lo >> 54)}; }
__device__ __forceinline__ Set128 dn10(Set128 a) { return Set128{(a.lo >> 10) | (a.hi << 54), a.hi >> 10}; }
// w (< 32) bits of x starting at square off (0 <= off < 128)
__device__ __forceinline__ uint32_t bits_at(Set128 x, int off, int w)
{
    const uint64_t v = off >= 64 ? (x.hi >> (off - 64)) : (off == 0 ? x.lo : ((x.lo >> off) | (x.hi << (64 - off))));
    return (uint32_t)v & ((1u << w) - 1u);
}

// From-square segments: lane j of a team of L lanes owns squares
// [W*j, W*j + W) (W = 25, 13, 7 or 4 squares for L = 4, 8, 16, 32).
template <int L> struct Seg {
    static constexpr int W = (kSquares + L - 1) / L;
    static constexpr int N = (kSquares + W - 1) / W;
    static_assert(N <= kSegMax && N <= L, "segments");
};

// ----------------------------------------------------------------- move generation
// Slides of the Scout on square s of player P: squares it can slide south,
// west, east and north, stopping before a lake or an own piece and on the
// first enemy piece (included).  occ: every piece; enm: the enemy pieces.
struct Runs {
    int ns, nw, ne, nn;
};
__device__ __forceinline__ Runs scout_runs(const SmemGame* G, int s, Set128 occ, Set128 enm)
{
    const int r = s / 10, c = s - 10 * r;
    const uint32_t rowocc = bits_at(occ, 10 * r, 10) | ((r == 4 || r == 5) ? kLakeRow : 0u);
    const uint32_t colocc = G->colocc[c] | ((c == 2 || c == 3 || c == 6 || c == 7) ? kLakeCol : 0u);
    // empty squares in each direction, then whether the blocker is an enemy
    // piece (its square is in enm; a lake is in neither set)
    const uint32_t e = rowocc >> (c + 1);
    const int runE = e ? __ffs(e) - 1 : 9 - c;
    const int capE = (e && test128(enm, s + runE + 1)) ? 1 : 0;
    const uint32_t w = rowocc & ((1u << c) - 1u);
    const int hw = w ? 31 - __clz(w) : -1;
    const int capW = (hw >= 0 && test128(enm, 10 * r + hw)) ? 1 : 0;
    const uint32_t n = colocc >> (r + 1);
    const int runN = n ? __ffs(n) - 1 : 9 - r;
    const int capN = (n && test128(enm, s + 10 * (runN + 1))) ? 1 : 0;
    const uint32_t so = colocc & ((1u << r) - 1u);
    const int hs = so ? 31 - __clz(so) : -1;
    const int capS = (hs >= 0 && test128(enm, 10 * hs + c)) ? 1 : 0;
    Runs R;
    R.ne = runE + capE;
    R.nw = c - 1 - hw + capW;
    R.nn = runN + capN;
    R.ns = r - 1 - hs + capS;
    return R;
}

// The destinations (a set over to-squares) of a Scout with slides R.
__device__ __forceinline__ Set128 scout_set(int s, const Runs& R)
{
    const int r = s / 10, c = s - 10 * r;
    Set128 d = or128(range128(s + 1, R.ne), range128(s - R.nw, R.nw));
    d = or128(d, column128(c, r + 1, r + R.nn));
    return or128(d, column128(c, r - R.ns, r - 1));
}

// Counts (and, if write_mask, records) the moves of player P; with mdst,
// also writes them as the 1,264-byte legal mask of the output layout to
// mdst (bit a&7 of byte a>>3 for action a = from*100 + to; the row is cleared
// first).  physical: movement rules only (App. A "Piece details"); otherwise
// the two-square and chasing rules filter as rule_flags says.  Team-uniform
// result.  The records are the moves per from-square (G->sq_cnt) and either
// a descriptor per from-square (G->desc; mdst, if any, is an output row in
// global memory) or, with kRows, the mask itself in mdst (a shared-memory
// buffer that the caller's selection reads; mdst is required then).
//
// Non-Scout moves come from four shifted square sets over the whole board;
// each lane records those of its own segment of from-squares.  A non-Scout's
// moves are one window of at most 21 mask bits (to-squares s-10, s-1, s+1,
// s+10 are bits 101s-10, 101s-1, 101s+1, 101s+10); two windows never share a
// 32-bit word, so an output row gets each with plain stores, before the
// Scouts' bits (shared-memory rows take atomic ORs throughout).  Scouts take
// one lane each; a Scout's row and column slides are written word by word
// with atomic ORs.  Moves that a rule may forbid (those of the piece under
// the two-square rule; all moves while a chase position can recur) go
// through filter_dests.
template <int L, bool kRows = false>
__device__ __noinline__ int gen_moves(SmemGame* G, Team<L>, int P, uint32_t rule_flags, bool physical,
                                      bool write_mask, const uint64_t* pi, uint32_t* mdst)
{
    const Team<L> T;
    constexpr int SW = Seg<L>::W;
    if constexpr (kRows) mdst = rows_of(G);   // row mode: the mask follows the record (mdst is ignored)
    if (!write_mask) mdst = nullptr;
    if (write_mask) {
        if constexpr (kRows) {
            // the per-square counts and the mask: one run of 16-byte words
            constexpr int kZero = (kCntBytes + kMaskBytes) / 16;
            uint4* z = reinterpret_cast<uint4*>(G->sq_cnt);
#pragma unroll
            for (int k = 0; k < (kZero + L - 1) / L; ++k) {
                const int i = T.tl + k * L;
                if (i < kZero) z[i] = make_uint4(0, 0, 0, 0);
            }
        } else {
            uint4* z = reinterpret_cast<uint4*>(G->sq_cnt);
            for (int i = T.tl; i < kCntBytes / 16; i += L) z[i] = make_uint4(0, 0, 0, 0);
            if (mdst) {
                uint4* m4 = reinterpret_cast<uint4*>(mdst);
#pragma unroll
                for (int k = 0; k < (kMaskBytes / 16 + L - 1) / L; ++k) {
                    const int i = T.tl + k * L;
                    if (i < kMaskBytes / 16) m4[i] = make_uint4(0, 0, 0, 0);
                }
            }
        }
    }
    const int ts_pid = G->c.ts_pid[P];
    const bool ts_on = !physical && (rule_flags & kTwoSquare) && ts_pid != kNone && G->c.ts_len[P] == 4 &&
                       (G->c.flags[ts_pid] & 1);
    const int ts_from = ts_on ? G->c.sq[ts_pid] : -1;
    const bool chase_on = !physical && (rule_flags & kChase) && G->c.chaser == P && G->c.n_pi > 0 &&
                          chase_live(G, T, pi, P);
    if (!kRows && write_mask && T.leader()) G->gen_chase = chase_on ? 1 : 0;
    const PlyCtx x = make_ctx(G);
    T.sync();   // counts and mask row cleared before anything is recorded
    const Set128 own = ld128(G->bocc[P]), enm = ld128(G->bocc[1 - P]), mv = ld128(G->bmov[P]);
    // empty or enemy squares
    const Set128 fre{~own.lo & ~kLakesLo, ~own.hi & kValidHi};
    const Set128 FE = and128(and128(mv, dn1(fre)), Set128{~kCol9Lo, ~kCol9Hi});
    const Set128 FW = and128(and128(mv, up1(fre)), Set128{~kCol0Lo, ~kCol0Hi});
    const Set128 FN = and128(mv, dn10(fre));
    const Set128 FS = and128(mv, up10(fre));
    const int off = SW * T.tl;
    uint32_t fe = bits_at(FE, off, SW), fw = bits_at(FW, off, SW);
    uint32_t fn = bits_at(FN, off, SW), fs = bits_at(FS, off, SW);
    uint32_t moving = fe | fw | fn | fs;
    int cnt = 0;
    if (chase_on) {
        while (moving) {
            const int c = __ffs(moving) - 1;
            moving &= moving - 1;
            const int s = off + c;
            Set128 d{0ull, 0ull};
            if ((fs >> c) & 1u) d = or128(d, bit128(s - 10));
            if ((fw >> c) & 1u) d = or128(d, bit128(s - 1));
            if ((fe >> c) & 1u) d = or128(d, bit128(s + 1));
            if ((fn >> c) & 1u) d = or128(d, bit128(s + 10));
            d = filter_dests(G, P, s, s == ts_from, true, x, pi, d);
            const int k = popc128(d);
            cnt += k;
            if (write_mask && k) {
                G->sq_cnt[s] = (uint8_t)k;
                if (!kRows)
                    G->desc[s] = (uint16_t)(kDescStep | (s >= 10 && test128(d, s - 10) ? 1u : 0u) |
                                            (s >= 1 && test128(d, s - 1) ? 2u : 0u) | (test128(d, s + 1) ? 4u : 0u) |
                                            (test128(d, s + 10) ? 8u : 0u));
                if (mdst) or_row(mdst, s, d);
            }
        }
    } else {
        // the piece under the two-square rule (if in this segment) is the only
        // one whose destinations need a filter
        const uint32_t ts_bit = (ts_from >= off && ts_from < off + SW) ? (1u << (ts_from - off)) : 0u;
        if (moving & ts_bit) {
            const int c = ts_from - off, s = ts_from;
            Set128 d{0ull, 0ull};
            if ((fs >> c) & 1u) d = or128(d, bit128(s - 10));
            if ((fw >> c) & 1u) d = or128(d, bit128(s - 1));
            if ((fe >> c) & 1u) d = or128(d, bit128(s + 1));
            if ((fn >> c) & 1u) d = or128(d, bit128(s + 10));
            d = filter_dests(G, P, s, true, false, x, pi, d);
            const int k = popc128(d);
            cnt += k;
            if (write_mask && k) {
                G->sq_cnt[s] = (uint8_t)k;
                if (!kRows)
                    G->desc[s] = (uint16_t)(kDescStep | (s >= 10 && test128(d, s - 10) ? 1u : 0u) |
                                            (s >= 1 && test128(d, s - 1) ? 2u : 0u) | (test128(d, s + 1) ? 4u : 0u) |
                                            (test128(d, s + 10) ? 8u : 0u));
                if (mdst) or_row(mdst, s, d);
            }
            moving &= ~ts_bit;
            fe &= ~ts_bit; fw &= ~ts_bit; fn &= ~ts_bit; fs &= ~ts_bit;
        }
        cnt += __popc(fe) + __popc(fw) + __popc(fn) + __popc(fs);
        if (write_mask) {
            while (moving) {
                const int c = __ffs(moving) - 1;
                moving &= moving - 1;
                const int s = off + c;
                if constexpr (kRows) {
                    uint32_t pat = ((fs >> c) & 1u) | (((fw >> c) & 1u) << 9) | (((fe >> c) & 1u) << 11) |
                                   (((fn >> c) & 1u) << 20);
                    G->sq_cnt[s] = (uint8_t)__popc(pat);
                    int base = 101 * s - 10;
                    if (s == 0) { pat >>= 10; base = 0; }   // square 0 has no south or west move
                    const uint64_t v = (uint64_t)pat << (base & 31);
                    atomicOr(&mdst[base >> 5], (uint32_t)v);
                    if (v >> 32) atomicOr(&mdst[(base >> 5) + 1], (uint32_t)(v >> 32));
                } else {
                    const uint32_t dirs = ((fs >> c) & 1u) | (((fw >> c) & 1u) << 1) | (((fe >> c) & 1u) << 2) |
                                          (((fn >> c) & 1u) << 3);
                    G->sq_cnt[s] = (uint8_t)__popc(dirs);
                    G->desc[s] = (uint16_t)(kDescStep | dirs);
                    if (mdst) {
                        uint32_t pat = (dirs & 1u) | ((dirs & 2u) << 8) | ((dirs & 4u) << 9) | ((dirs & 8u) << 17);
                        int base = 101 * s - 10;
                        if (s == 0) { pat >>= 10; base = 0; }   // square 0 has no south or west move
                        const uint64_t v = (uint64_t)pat << (base & 31);
                        mdst[base >> 5] = (uint32_t)v;
                        if (v >> 32) mdst[(base >> 5) + 1] = (uint32_t)(v >> 32);
                    }
                }
            }
        }
    }
    if (!kRows && mdst) T.sync();   // the windows are in place before the Scouts' bits are ORed in
    // Scouts, one per lane
    const Set128 occ{own.lo | enm.lo, own.hi | enm.hi};
    for (int si = T.tl; si < 8; si += L) {
        const int spid = G->scout_pid[P][si];
        if (spid != kNone && (G->c.flags[spid] & 1)) {
            const int s = G->c.sq[spid];
            const Runs R = scout_runs(G, s, occ, enm);
            int cnt_sc = R.ne + R.nw + R.nn + R.ns;
            if (cnt_sc && (chase_on || s == ts_from)) {
                const Set128 d = filter_dests(G, P, s, s == ts_from, chase_on, x, pi, scout_set(s, R));
                cnt_sc = popc128(d);
                if (write_mask && cnt_sc) {
                    if (!kRows) G->desc[s] = kDescFiltered;
                    if (mdst) or_row(mdst, s, d);
                }
            } else if (cnt_sc && write_mask) {
                if (!kRows) G->desc[s] = (uint16_t)(R.ns | (R.nw << 4) | (R.ne << 8) | (R.nn << 12));
                if (mdst) {
                    // mask bits 101s+j (row, j in [-nw, ne]) and 101s+10k (column,
                    // k in [-ns, nn]), j, k != 0, word by word: the column bits are
                    // the bits of [101s-10ns, 101s+10nn] equal to s, so to c, modulo
                    // 10, in word w the bits (c - 2w) mod 10 + 10i (32 = 2 mod 10)
                    const int c = s - 10 * (s / 10);
                    const int ctr = 101 * s;
                    const int clo = ctr - 10 * R.ns, chi = ctr + 10 * R.nn, rlo = ctr - R.nw, rhi = ctr + R.ne;
                    const int wlo = min(clo, rlo) >> 5, whi = max(chi, rhi) >> 5;
                    int m = (c + 640 - 2 * wlo) % 10;
                    // kept rolled: the unrolled copies cost more in instruction
                    // fetch than the loop's branches
#pragma unroll 1
                    for (int wi = wlo; wi <= whi; ++wi) {
                        const int b0 = 32 * wi;
                        uint32_t v = ((0x40100401u << m) & range32(clo - b0, chi - b0)) | range32(rlo - b0, rhi - b0);
                        if (ctr >= b0 && ctr < b0 + 32) v &= ~(1u << (ctr - b0));
                        if (v) atomicOr(&mdst[wi], v);
                        m = m >= 2 ? m - 2 : m + 8;
                    }
                }
            }
            if (write_mask && cnt_sc) G->sq_cnt[s] = (uint8_t)cnt_sc;
            cnt += cnt_sc;
        }
    }
    const int total = T.sum(cnt);
    T.sync();
    return total;
}

// The destinations of the piece on from-square s of the player to move, as
// the last generation recorded them: the k-th (ascending) of its G->sq_cnt[s]
// moves.  A Scout whose moves a rule filters has them rebuilt (same inputs as
// at generation: nothing moved since).
__device__ __forceinline__ int kth_dest(const SmemGame* G, int s, int k, const uint64_t* pi, uint32_t rule_flags)
{
    const uint32_t d = G->desc[s];
    if ((d & kDescStep) == kDescStep) {
        const int b = nth_set_bit(d & 0xFu, k);   // 0 south, 1 west, 2 east, 3 north
        return s + (b == 0 ? -10 : b == 1 ? -1 : b == 2 ? 1 : 10);
    }
    if (d != kDescFiltered) {
        const int ns = d & 15, nw = (d >> 4) & 15, ne = (d >> 8) & 15;
        if (k < ns) return s - 10 * (ns - k);
        k -= ns;
        if (k < nw) return s - nw + k;
        k -= nw;
        if (k < ne) return s + 1 + k;
        return s + 10 * (k - ne + 1);
    }
    const int P = G->c.ply & 1;
    const Set128 own = ld128(G->bocc[P]), enm = ld128(G->bocc[1 - P]);
    const int ts_pid = G->c.ts_pid[P];
    const bool ts_here = (rule_flags & kTwoSquare) && ts_pid != kNone && G->c.ts_len[P] == 4 &&
                         (G->c.flags[ts_pid] & 1) && G->c.sq[ts_pid] == s;
    const Set128 ds = filter_dests(G, P, s, ts_here, G->gen_chase != 0, make_ctx(G), pi,
                                   scout_set(s, scout_runs(G, s, Set128{own.lo | enm.lo, own.hi | enm.hi}, enm)));
    const int nlo = __popcll(ds.lo);
    return k < nlo ? nth_set_bit64(ds.lo, k) : 64 + nth_set_bit64(ds.hi, k - nlo);
}

// Is action a among the legal moves the last generation recorded?
__device__ __forceinline__ bool move_recorded(const SmemGame* G, int a, const uint64_t* pi, uint32_t rule_flags)
{
    if (a < 0 || a >= 10000) return false;
    const int s = a / 100, to = a - 100 * s;
    const int n = G->sq_cnt[s];
    for (int k = 0; k < n; ++k)
        if (kth_dest(G, s, k, pi, rule_flags) == to) return true;
    return false;
}

// Clears a 1,264-byte mask row (the mask of a player without moves).
template <int L>
__device__ __forceinline__ void zero_row(uint32_t* mdst, const Team<L>& T)
{
    if (mdst) {
        uint4* m4 = reinterpret_cast<uint4*>(mdst);
        for (int i = T.tl; i < kMaskBytes / 16; i += L) m4[i] = make_uint4(0, 0, 0, 0);
    }
}

// The four mask words holding from-square s's row (actions 100s .. 100s+99),
// bits of the neighbouring rows cleared; returns the row's first word index.
__device__ __forceinline__ int row_words(const uint32_t* mask, int s, uint32_t r[4])
{
    const int b = 100 * s, w = b >> 5, off = b & 31;   // off = 4s mod 32: 0 .. 28
    const int hb = off + 4;                             // row bits in the fourth word
    r[0] = mask[w] & (~0u << off);
    r[1] = mask[w + 1];
    r[2] = mask[w + 2];
    r[3] = mask[w + 3] & (hb >= 32 ? ~0u : ((1u << hb) - 1u));
    return w;
}

// The idx-th legal action (ascending action order) of the player to move;
// team-uniform result.  Lane t owns squares [Q*t, Q*t + Q) (Q = 128 / L) and
// sums their move counts from G->sq_cnt; a scan over the team finds the lane
// holding move idx, that lane finds the square (per-byte prefix sums of its
// count words) and then the move among the square's own: from the square's
// mask row (row mode, rows_of) or from its descriptor (kth_dest).
template <int L, bool kRows>
__device__ __forceinline__ int select_impl(const SmemGame* G, uint32_t idx, const uint64_t* pi, uint32_t rule_flags)
{
    const Team<L> T;
    constexpr int NW = kCntBytes / L / 4;   // count words per lane: 8, 4, 2, 1
    const int t = T.tl;
    uint32_t w[NW];
    if constexpr (NW >= 4) {
        const uint4* c4 = reinterpret_cast<const uint4*>(G->sq_cnt) + (NW / 4) * t;
#pragma unroll
        for (int j = 0; j < NW / 4; ++j) {
            const uint4 v = c4[j];
            w[4 * j] = v.x; w[4 * j + 1] = v.y; w[4 * j + 2] = v.z; w[4 * j + 3] = v.w;
        }
    } else if constexpr (NW == 2) {
        const uint2 v = reinterpret_cast<const uint2*>(G->sq_cnt)[t];
        w[0] = v.x; w[1] = v.y;
    } else {
        w[0] = reinterpret_cast<const uint32_t*>(G->sq_cnt)[t];
    }
    int sum = 0;
#pragma unroll
    for (int j = 0; j < NW; ++j) sum = (int)__dp4a(w[j], 0x01010101u, (unsigned)sum);
    int incl = sum;
#pragma unroll
    for (int o = 1; o < L; o <<= 1) {
        const int v = __shfl_up_sync(T.mask, incl, o, L);
        if (t >= o) incl += v;
    }
    const uint32_t own = T.ballot((int)idx >= incl - sum && (int)idx < incl);
    int a = -1;
    if (own & (1u << t)) {
        int k = (int)idx - (incl - sum);
        // the count word holding move k
        int j = 0;
        uint32_t wj = w[0];
#pragma unroll
        for (int i = 0; i < NW; ++i) {
            const int ci = (int)__dp4a(w[i], 0x01010101u, 0u);
            if (j == i && k >= ci && i + 1 < NW) { k -= ci; j = i + 1; wj = w[i + 1]; }
        }
        // the square within it: byte b of pre is the sum of bytes 0..b (at
        // most 4 x 18 moves, no carries), the first byte above k holds move k
        const uint32_t pre = wj * 0x01010101u;
        const int b = (__ffs(__vcmpgtu4(pre, 0x01010101u * (uint32_t)k)) - 1) >> 3;
        if (b > 0) k -= (int)((pre >> (8 * (b - 1))) & 0xFFu);
        const int s = 4 * (NW * t + j) + b;
        if constexpr (kRows) {
            uint32_t r[4];
            const int w0 = row_words(rows_of(G), s, r);
            int i = 0;
            while (i < 3 && k >= __popc(r[i])) { k -= __popc(r[i]); ++i; }
            a = 32 * (w0 + i) + nth_set_bit(r[i], k);
        } else {
            a = 100 * s + kth_dest(G, s, k, pi, rule_flags);
        }
    }
    return T.shfl(a, own ? __ffs(own) - 1 : 0);
}

// The magnet policy's move (Tab. notation rho) for the player to move:
// piece number uniform_below(w0, pieces with a legal move) in ascending
// square order, then move number uniform_below(w1, its moves) in ascending
// action order.  Lane t looks at the squares [Q*t, Q*t + Q) of G->sq_cnt
// (Q = 128 / L).  Team-uniform result.
template <int L>
__device__ __forceinline__ int magnet_impl(const SmemGame* G, uint32_t w0, uint32_t w1, const uint64_t* pi,
                                           uint32_t rule_flags)
{
    const Team<L> T;
    constexpr int NW = kCntBytes / L / 4;
    const int t = T.tl;
    // bit i: square 4*NW*t + i has a legal move
    uint32_t live = 0;
    const uint32_t* cw = reinterpret_cast<const uint32_t*>(G->sq_cnt) + NW * t;
#pragma unroll
    for (int j = 0; j < NW; ++j) {
        const uint32_t v = cw[j];
#pragma unroll
        for (int b = 0; b < 4; ++b)
            if ((v >> (8 * b)) & 0xFFu) live |= 1u << (4 * j + b);
    }
    const int np = __popc(live);
    int incl = np;
#pragma unroll
    for (int o = 1; o < L; o <<= 1) {
        const int v = __shfl_up_sync(T.mask, incl, o, L);
        if (t >= o) incl += v;
    }
    const int pieces = T.shfl(incl, L - 1);
    const int want = (int)uniform_below(w0, (uint32_t)pieces);
    const uint32_t own_lane = T.ballot(want >= incl - np && want < incl);
    int a = -1;
    if (own_lane & (1u << t)) {
        const int s = 4 * NW * t + nth_set_bit(live, want - (incl - np));
        const int k = (int)uniform_below(w1, (uint32_t)G->sq_cnt[s]);
        a = 100 * s + kth_dest(G, s, k, pi, rule_flags);
    }
    return T.shfl(a, own_lane ? __ffs(own_lane) - 1 : 0);
}

template <int L, bool kRows = false>
__device__ __noinline__ int select_action(const SmemGame* G, Team<L>, uint32_t idx, const uint64_t* pi,
                                          uint32_t rule_flags)
{
    return select_impl<L, kRows>(G, idx, pi, rule_flags);
}

// Is the flag of `side` captured?
__device__ __forceinline__ bool flag_dead(const SmemGame* G, int side)
{
    return !(G->c.flags[G->flag_pid[side]] & 1);
}

// ----------------------------------------------------------------- apply
// Plays action a for the player to move.  ring/pi: this game's history ring
// and chase-position store.
template <int L>
__device__ __forceinline__ void apply_impl(SmemGame* G, int a, uint16_t* ring, uint64_t* pi)
{
    const Team<L> T;
    if (T.leader() && a >= 0 && a < 10000) {
        const PlyCtx x = make_ctx(G);
        GameCore& c = G->c;
        const int P = c.ply & 1;
        const int from = a / 100, to = a - 100 * (a / 100);
        const int X = G->board[from];
        const int cls = classify(G, x, P, from, to);
        const int rf = from / 10, cf = from - 10 * rf, rt = to / 10, ct = to - 10 * rt;
        const int dist = rf == rt ? abs(cf - ct) : abs(rf - rt);
        uint8_t fx = c.flags[X];
        if (dist > 1) fx |= 8;
        fx |= 4;
        const bool battle = G->board[to] != kEmpty;
        uint64_t h = c.hash_side[P] ^ zkey(X, from);   // mover's pieces
        uint64_t hq = c.hash_side[1 - P];               // the other side's pieces
        int D = -1;
        bool d_died = false, x_alive = true;
        const int tX = c.type[X];
        uint64_t* kindX = tX == kScout ? G->bsco[P] : G->bmov[P];
        G->board[from] = kEmpty;
        bb_clr(G->bocc[P], from);
        bb_clr(kindX, from);
        G->colocc[cf] &= (uint16_t)~(1u << rf);
        if (!battle) {
            G->board[to] = (uint8_t)X;
            c.sq[X] = (uint8_t)to;
            h ^= zkey(X, to);
        } else {
            D = G->board[to];
            uint8_t fd = c.flags[D];
            const bool d_rev = fd & 2;
            const int td = c.type[D];
            // Tab. pieces: Flag loses to any attacker; Bomb beats all but the
            // Miner; the attacking Spy beats the Marshal; otherwise by rank.
            int out;
            if (td == kFlag) out = 1;
            else if (td == kBomb) out = tX == kMiner ? 1 : 2;
            else if (tX == kSpy && td == kMarshal) out = 1;
            else out = tX > td ? 1 : (tX < td ? 2 : 3);
            fx |= 2;
            fd |= 2;
            if (out == 1) {
                fd = (uint8_t)((fd & 0x0E) | ((d_rev ? 4 : 6) << 4));
                d_died = true;
                G->board[to] = (uint8_t)X;
                c.sq[X] = (uint8_t)to;
                h ^= zkey(X, to);
                hq ^= zkey(D, to);
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
                hq ^= zkey(D, to);
            }
            c.flags[D] = fd;
            if (d_died) {
                const int Q = 1 - P;
                bb_clr(G->bocc[Q], to);
                bb_clr(G->bmov[Q], to);
                bb_clr(G->bsco[Q], to);
            }
        }
        if (x_alive) {
            bb_set(G->bocc[P], to);
            bb_set(kindX, to);
        }
        if (G->board[to] != kEmpty) G->colocc[ct] |= (uint16_t)(1u << rt);
        else G->colocc[ct] &= (uint16_t)~(1u << rt);
        c.flags[X] = fx;
        c.hash_side[P] = h;
        c.hash_side[1 - P] = hq;
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
            if (c.n_pi < kPiCap) {
                pi[2 * c.n_pi] = h; pi[2 * c.n_pi + 1] = hq;
                G->pi_theirs[c.n_pi & 3] = hq;
                G->pi_mine[c.n_pi & 3] = h;
                c.n_pi += 1;
            }
            c.chase_plies += 1;
        } else if (cls == kClEvade && c.chaser == 1 - P) {
            c.chase_plies += 1;
        } else {
            c.chaser = kNone; c.n_pi = 0; c.chase_plies = 0;
        }
        if (ring) ring[ply_before & (kRing - 1)] = (uint16_t)a;
        G->h1 = G->h0;
        G->h0 = (uint16_t)a;
    }
    T.sync();
}

// The same move in two halves, for kernels whose other warps read the
// position while the move is worked out (the replay): plan_apply reads
// every input and computes the new state in registers without writing;
// commit_apply writes it.  Together they make exactly the changes of
// apply_impl.
struct ApplyPlan {
    int a, from, to, X, D, to_after, cls, ply, battleless, h0;
    int cf, ct;
    uint32_t vf, vt;              // new column occupancy of the from- and to-columns
    bool battle, x_alive, d_died, scout;
    uint8_t fx, fd;
    uint64_t h, hq;
    Set128 occP, kindP, occQ, movQ, scoQ;
    int ts_mode, ts_len, s1, s2, s3;   // 0 reset, 1 shift in `to`, 2 append `to`, 3 new piece
    bool ts_reset_q;
    int chaser, n_pi, chase_plies;
};

__device__ __forceinline__ ApplyPlan plan_apply(const SmemGame* G, int a)
{
    ApplyPlan q;
    const GameCore& c = G->c;
    q.a = a;
    const int from = a / 100, to = a - 100 * (a / 100);
    q.from = from; q.to = to;
    const int rf = from / 10, cf = from - 10 * rf, rt = to / 10, ct = to - 10 * rt;
    q.cf = cf; q.ct = ct;
    const int ply = c.ply;
    q.ply = ply;
    const int P = ply & 1, Q = 1 - P;
    const int X = G->board[from];
    const int D = G->board[to];
    const int h0 = G->h0;
    q.h0 = h0;
    const int prev_to = h0 == 0xFFFF ? -1 : h0 % 100;
    const uint8_t on_prev = prev_to >= 0 ? G->board[prev_to] : kEmpty;
    const uint8_t nS = rt > 0 ? G->board[to - 10] : kEmpty;
    const uint8_t nN = rt < 9 ? G->board[to + 10] : kEmpty;
    const uint8_t nW = ct > 0 ? G->board[to - 1] : kEmpty;
    const uint8_t nE = ct < 9 ? G->board[to + 1] : kEmpty;
    const bool prev_nb = !c.last_battle;
    q.battleless = c.battleless;
    const uint64_t hsP = c.hash_side[P], hsQ = c.hash_side[Q];
    const Set128 occP = ld128(G->bocc[P]), occQ = ld128(G->bocc[Q]);
    const Set128 movP = ld128(G->bmov[P]), scoP = ld128(G->bsco[P]);
    const Set128 movQ = ld128(G->bmov[Q]), scoQ = ld128(G->bsco[Q]);
    const uint32_t col_f = G->colocc[cf], col_t = G->colocc[ct];
    const int ts_pidP = c.ts_pid[P], ts_lenP = c.ts_len[P], ts_pidQ = c.ts_pid[Q];
    q.s1 = c.ts_sq[P][1]; q.s2 = c.ts_sq[P][2]; q.s3 = c.ts_sq[P][3];
    q.chaser = c.chaser; q.n_pi = c.n_pi; q.chase_plies = c.chase_plies;
    const bool battle = D != kEmpty;
    const int Dp = battle ? D : X;   // the defender, or any valid piece
    const uint8_t fX0 = c.flags[X], fD0 = c.flags[Dp];
    const int tX = c.type[X], tD = c.type[Dp];
    q.X = X; q.D = D; q.battle = battle;
    if (battle) q.cls = kClBattle;
    else if (prev_to >= 0 && prev_nb && enemy_of(on_prev, P) && adjacent(from, prev_to) && !adjacent(to, prev_to))
        q.cls = kClEvade;
    else
        q.cls = (enemy_of(nS, P) || enemy_of(nN, P) || enemy_of(nW, P) || enemy_of(nE, P)) ? kClThreat : kClQuiet;
    const uint64_t zXf = zkey(X, from), zXt = zkey(X, to), zDt = zkey(Dp, to);
    const int dist = rf == rt ? abs(cf - ct) : abs(rf - rt);
    uint8_t fx = (uint8_t)(fX0 | 4 | (dist > 1 ? 8 : 0));
    uint8_t fd = fD0;
    bool d_died = false, x_alive = true;
    int to_after = X;
    if (battle) {
        const bool d_rev = fD0 & 2;
        int out;
        if (tD == kFlag) out = 1;
        else if (tD == kBomb) out = tX == kMiner ? 1 : 2;
        else if (tX == kSpy && tD == kMarshal) out = 1;
        else out = tX > tD ? 1 : (tX < tD ? 2 : 3);
        fx |= 2;
        fd |= 2;
        if (out == 1) {
            fd = (uint8_t)((fd & 0x0E) | ((d_rev ? 4 : 6) << 4));
            d_died = true;
        } else if (out == 2) {
            fx = (uint8_t)((fx & 0x0E) | ((d_rev ? 1 : 3) << 4));
            x_alive = false;
            to_after = D;
        } else {
            fx = (uint8_t)((fx & 0x0E) | ((d_rev ? 2 : 3) << 4));
            fd = (uint8_t)((fd & 0x0E) | ((d_rev ? 5 : 6) << 4));
            d_died = true;
            x_alive = false;
            to_after = kEmpty;
        }
    }
    q.fx = fx; q.fd = fd; q.x_alive = x_alive; q.d_died = d_died; q.to_after = to_after;
    q.h = hsP ^ zXf ^ (x_alive ? zXt : 0ull);
    q.hq = hsQ ^ (d_died ? zDt : 0ull);
    const Set128 bf = bit128(from), bt = bit128(to);
    const Set128 add = x_alive ? bt : Set128{0ull, 0ull};
    q.scout = tX == kScout;
    const Set128 kind0 = q.scout ? scoP : movP;
    q.occP = Set128{(occP.lo & ~bf.lo) | add.lo, (occP.hi & ~bf.hi) | add.hi};
    q.kindP = Set128{(kind0.lo & ~bf.lo) | add.lo, (kind0.hi & ~bf.hi) | add.hi};
    q.occQ = Set128{occQ.lo & ~bt.lo, occQ.hi & ~bt.hi};
    q.movQ = Set128{movQ.lo & ~bt.lo, movQ.hi & ~bt.hi};
    q.scoQ = Set128{scoQ.lo & ~bt.lo, scoQ.hi & ~bt.hi};
    q.vf = col_f & ~(1u << rf);
    const uint32_t vt0 = cf == ct ? q.vf : col_t;
    q.vt = to_after != kEmpty ? (vt0 | (1u << rt)) : (vt0 & ~(1u << rt));
    if (!x_alive) q.ts_mode = 0;
    else if (ts_pidP == X && ts_lenP >= 2) q.ts_mode = ts_lenP == 4 ? 1 : 2;
    else q.ts_mode = 3;
    q.ts_len = ts_lenP;
    q.ts_reset_q = d_died && ts_pidQ == D;
    return q;
}

__device__ __forceinline__ void commit_apply(SmemGame* G, const ApplyPlan& q, uint16_t* ring, uint64_t* pi)
{
    GameCore& c = G->c;
    const int P = q.ply & 1, Q = 1 - P;
    G->board[q.from] = kEmpty;
    G->board[q.to] = (uint8_t)q.to_after;
    G->bocc[P][0] = q.occP.lo; G->bocc[P][1] = q.occP.hi;
    uint64_t* kindX = q.scout ? G->bsco[P] : G->bmov[P];
    kindX[0] = q.kindP.lo; kindX[1] = q.kindP.hi;
    if (q.d_died) {
        G->bocc[Q][0] = q.occQ.lo; G->bocc[Q][1] = q.occQ.hi;
        G->bmov[Q][0] = q.movQ.lo; G->bmov[Q][1] = q.movQ.hi;
        G->bsco[Q][0] = q.scoQ.lo; G->bsco[Q][1] = q.scoQ.hi;
    }
    if (q.cf != q.ct) G->colocc[q.cf] = (uint16_t)q.vf;
    G->colocc[q.ct] = (uint16_t)q.vt;
    c.sq[q.X] = (uint8_t)q.to;
    c.flags[q.X] = q.fx;
    if (q.battle) c.flags[q.D] = q.fd;
    c.hash_side[P] = q.h;
    c.hash_side[Q] = q.hq;
    c.battleless = q.battle ? 0 : (int16_t)(q.battleless + 1);
    c.last_battle = q.battle ? 1 : 0;
    c.ply = (int16_t)(q.ply + 1);
    if (q.ts_mode == 0) {
        c.ts_pid[P] = kNone; c.ts_len[P] = 0;
        c.ts_sq[P][0] = c.ts_sq[P][1] = c.ts_sq[P][2] = c.ts_sq[P][3] = kNone;
    } else if (q.ts_mode == 1) {
        c.ts_sq[P][0] = (uint8_t)q.s1; c.ts_sq[P][1] = (uint8_t)q.s2;
        c.ts_sq[P][2] = (uint8_t)q.s3; c.ts_sq[P][3] = (uint8_t)q.to;
    } else if (q.ts_mode == 2) {
        c.ts_sq[P][q.ts_len] = (uint8_t)q.to;
        c.ts_len[P] = (uint8_t)(q.ts_len + 1);
    } else {
        c.ts_pid[P] = (uint8_t)q.X; c.ts_len[P] = 2;
        c.ts_sq[P][0] = (uint8_t)q.from; c.ts_sq[P][1] = (uint8_t)q.to;
        c.ts_sq[P][2] = c.ts_sq[P][3] = kNone;
    }
    if (q.ts_reset_q) {
        c.ts_pid[Q] = kNone; c.ts_len[Q] = 0;
        c.ts_sq[Q][0] = c.ts_sq[Q][1] = c.ts_sq[Q][2] = c.ts_sq[Q][3] = kNone;
    }
    if (q.cls == kClThreat) {
        int n = q.n_pi, plies = q.chase_plies;
        if (q.chaser != P) { n = 0; plies = 0; }
        if (n < kPiCap) {
            pi[2 * n] = q.h; pi[2 * n + 1] = q.hq;
            G->pi_theirs[n & 3] = q.hq;
            G->pi_mine[n & 3] = q.h;
            n += 1;
        }
        c.chaser = (uint8_t)P;
        c.n_pi = (uint8_t)n;
        c.chase_plies = (uint8_t)(plies + 1);
    } else if (q.cls == kClEvade && q.chaser == Q) {
        c.chase_plies = (uint8_t)(q.chase_plies + 1);
    } else {
        c.chaser = kNone; c.n_pi = 0; c.chase_plies = 0;
    }
    if (ring) ring[q.ply & (kRing - 1)] = (uint16_t)q.a;
    G->h1 = (uint16_t)q.h0;
    G->h0 = (uint16_t)q.a;
}

template <int L>
__device__ __noinline__ void apply_move(SmemGame* G, Team<L>, int a, uint16_t* ring, uint64_t* pi)
{
    apply_impl<L>(G, a, ring, pi);
}

// The idx-th legal action (a < 0) or action a, then played: selection and
// the move in one call (the rollouts' ply).  Returns the action.
template <int L>
__device__ __noinline__ int select_apply(SmemGame* G, Team<L>, int a, uint32_t idx, uint16_t* ring, uint64_t* pi,
                                         uint32_t rule_flags)
{
    if (a < 0) a = select_impl<L, false>(G, idx, pi, rule_flags);
    apply_impl<L>(G, a, ring, pi);
    return a;
}

// The magnet policy's move for Philox words (w0, w1), then played.
template <int L>
__device__ __noinline__ int magnet_apply(SmemGame* G, Team<L>, uint32_t w0, uint32_t w1, uint16_t* ring, uint64_t* pi,
                                         uint32_t rule_flags)
{
    const int a = magnet_impl<L>(G, w0, w1, pi, rule_flags);
    apply_impl<L>(G, a, ring, pi);
    return a;
}

// ----------------------------------------------------------------- new game
// setup: custom types per piece id, or nullptr for the Philox setup of
// (slot, episode).
template <int L>
__device__ __noinline__ void reset_game(SmemGame* G, Team<L>, uint32_t k0, uint32_t k1, uint32_t slot,
                                        uint32_t episode, const uint8_t* setup)
{
    const Team<L> T;
    for (int p = T.tl; p < kPieces; p += L) {
        G->c.type[p] = setup ? setup[p] : sorted_type(p % 40);
        G->c.sq[p] = (uint8_t)start_square(p);
        G->c.flags[p] = 1;
    }
    T.sync();
    if (!setup && T.tl < 2) {
        uint8_t* arr = G->c.type + 40 * T.tl;
        uint4 w = make_uint4(0, 0, 0, 0);
        for (int i = 39; i >= 1; --i) {
            const int d = 39 - i;
            if ((d & 3) == 0)
                w = philox(make_uint4(slot, episode, 0u, (1u << 24) | ((uint32_t)T.tl << 8) | (uint32_t)(d >> 2)),
                           k0, k1);
            const uint32_t r = (d & 3) == 0 ? w.x : (d & 3) == 1 ? w.y : (d & 3) == 2 ? w.z : w.w;
            const uint32_t j = uniform_below(r, (uint32_t)(i + 1));
            const uint8_t t = arr[i];
            arr[i] = arr[j];
            arr[j] = t;
        }
    }
    if (T.leader()) {
        GameCore& c = G->c;
        c.ply = 0; c.battleless = 0; c.last_battle = 0;
        c.chaser = kNone; c.chase_plies = 0; c.n_pi = 0;
        c.ts_pid[0] = c.ts_pid[1] = kNone; c.ts_len[0] = c.ts_len[1] = 0;
        for (int i = 0; i < 4; ++i) c.ts_sq[0][i] = c.ts_sq[1][i] = kNone;
        c.terminated = 0; c.episode = episode; c.n_legal = 0;
    }
    T.sync();
    const uint64_t h0 = side_hash(G, T, 0), h1 = side_hash(G, T, 1);
    if (T.leader()) { G->c.hash_side[0] = h0; G->c.hash_side[1] = h1; }
    build_board(G, T);
    derive_state(G, (const uint16_t*)nullptr, (const uint64_t*)nullptr, T);
}

// ----------------------------------------------------------------- endings
struct PlyResult {
    int action;
    int code;
    int winner;
    int ply_idx;
};

// Ending after the ply just played (App. A "Game Summary", App. D.1); also
// records the moves of the player to move (G->sq_cnt, G->desc; their mask in
// mdst when given) and their count in n.  A captured flag ends the game
// before any move is recorded.
template <int L, bool kRows = false>
__device__ __forceinline__ void check_end(SmemGame* G, const Team<L>& T, const Rules& R, const uint64_t* pi,
                                          int& code, int& winner, int& n, uint32_t* mdst)
{
    const int Q = G->c.ply & 1, P = 1 - Q;
    code = 0;
    winner = -1;
    n = 0;
    if (flag_dead(G, Q)) {
        code = 1;
        winner = P;
    } else {
        n = gen_moves<L, kRows>(G, T, Q, R.flags, false, true, pi, mdst);
        if (n == 0) {
            const int phys = gen_moves<L, false>(G, T, P, R.flags, true, false, pi, (uint32_t*)nullptr);
            code = phys == 0 ? 3 : 2;
            winner = phys == 0 ? -1 : P;
        } else if (G->c.battleless >= R.k) {
            code = 4;
        } else if (G->c.ply >= R.cap) {
            code = 5;
        }
    }
    // Every lane has read the state the ending depends on before any lane
    // goes on to change it (a restart or the next rollout rewrites the game
    // record): without this barrier a lane that lags could read the new game
    // and take a different ending than its team, and the team's lanes would
    // then meet at different collectives.
    T.sync();
}

// The acting player of a fresh position has no legal move (n == 0).
template <int L>
__device__ __forceinline__ void start_end(SmemGame* G, const Team<L>& T, const Rules& R, const uint64_t* pi, int& code,
                                          int& winner)
{
    const int P = G->c.ply & 1;
    const int phys = gen_moves<L, false>(G, T, 1 - P, R.flags, true, false, pi, (uint32_t*)nullptr);
    code = phys == 0 ? 3 : 2;
    winner = phys == 0 ? -1 : 1 - P;
}

}  // namespace stg
