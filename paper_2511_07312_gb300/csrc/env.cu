// env.cu -- the batched environment (App. B.1 StrategoRolloutBuffer as a
// simulator): N independent game slots kept in HBM, stepped one ply per
// launch (st_env_step, the plain path) or many plies per persistent launch
// (st_env_run), with auto-reset, snapshots and per-slot counters.  The
// persistent launch runs 1, 2, 4 or 8 games per warp (teams of 32, 16, 8 or
// 4 lanes), the shape chosen by st_env_set_launch.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>
#include "rollout.cuh"
#include "host_common.h"

using namespace stg;

struct st_env {
    int device = 0;
    cudaStream_t stream = nullptr;
    int N = 0;
    uint64_t seed = 0;
    Rules rules{};
    GameCore* core = nullptr;
    uint16_t* ring = nullptr;
    uint64_t* pi = nullptr;
    uint32_t* stats = nullptr;
    int32_t* status = nullptr;      // [0] latched st_status, [1] first slot (min)
    int32_t* queue = nullptr;       // work counter of the persistent launch
    int32_t* part_done = nullptr;   // [N] parts of each slot played in the current persistent launch
    int wpb = 4, bps = 0, gpf = 1;  // launch shape of st_env_run
    int gpw = 1;                    // games per warp (1, 2, 4 or 8)
    int sms = 0;
    int max_bps = 0;
    cudaGraphExec_t graph = nullptr;
    int64_t graph_key[11] = {0};
    uint8_t* pool = nullptr;        // [2][pool_m][40] setups per side, or null
    int pool_m = 0;
    uint32_t pool_flags = 0;
    int32_t* pin_of = nullptr;      // [N] pinned record of each slot, -1 none
    RootState* pins = nullptr;      // [n_pins] pinned restart positions
    int n_pins = 0;
    long long now = 0;              // env steps taken (every slot advances one ply per step)
    uint32_t* hist = nullptr;       // [H][N] history ring (see hist_after)
    int H = 0;
    long long* d_now = nullptr;     // device copy of `now` while the history is on
    long long hist_start = 0;       // first step recorded
    long long cfg_floor = 0;        // last change of the reset sources
};

namespace stg {

static thread_local std::string g_err;

void set_error(const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
}

int sm_count()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n;
}

}  // namespace stg

extern "C" const char* st_last_error(void) { return stg::g_err.c_str(); }
extern "C" const char* st_version(void) { return "stratego-gb300 0.2 (sm_103a)"; }

namespace {

// Where new games come from besides the Philox setup.
struct ResetSrc {
    const uint8_t* pool;      // setup pool [2][pool_m][40], or null
    const int32_t* pin_of;    // [N] pinned record per slot (-1 none), null while nothing is pinned
    const RootState* pins;
    int pool_m;
    uint32_t pool_flags;
};

struct EnvArgs {
    GameCore* core;
    uint16_t* ring;
    uint64_t* pi;
    uint32_t* stats;
    int32_t* status;
    int N;
    uint32_t k0, k1;
    Rules R;
    ResetSrc reset;
    uint32_t* hist;           // history ring [H][N], or null
    const long long* now;     // steps taken before this launch
    int H;
};

__device__ __forceinline__ void latch(int32_t* status, int code, int slot)
{
    atomicCAS(&status[0], 0, code);
    atomicMin(&status[1], slot);
}

// The persistent step renders each ply's mask into a per-team staging
// buffer in shared memory and writes it to its ring row with one bulk
// asynchronous copy (TMA) issued by the team's first lane; the copy runs
// while the team selects and plays the next move (selection reads the move
// records, not the mask), and the buffer is not written again before
// mask_free.  Both addresses and the size are multiples of 16 bytes (the
// buffers sit at 16-byte offsets of the dynamic shared memory; ring rows are
// 1,264 bytes apart from a 256-byte-aligned base).
template <int L>
__device__ __forceinline__ void write_mask_async(const uint32_t* staged, const Team<L>& T, uint8_t* dst)
{
    // the lanes' mask writes (generic proxy) become visible to the copy engine
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    T.sync();
    if (T.leader()) {
        const uint32_t src = static_cast<uint32_t>(__cvta_generic_to_shared(staged));
        asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;"
                     :: "l"(dst), "r"(src), "r"((uint32_t)kMaskBytes) : "memory");
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    }
}

// Before the staging buffer is written again: the leader waits until its
// copies have read it.
template <int L>
__device__ __forceinline__ void mask_free(const Team<L>& T)
{
    if (T.leader()) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    T.sync();
}

__device__ __forceinline__ bool setup_counts_ok(const uint8_t* s)
{
    int cnt[2][12];
    for (int a = 0; a < 2; ++a)
        for (int t = 0; t < 12; ++t) cnt[a][t] = 0;
    for (int p = 0; p < 80; ++p) {
        if (s[p] >= 12) return false;
        cnt[p / 40][s[p]]++;
    }
    const int want[12] = {1, 8, 5, 4, 4, 4, 3, 2, 1, 1, 1, 6};
    for (int a = 0; a < 2; ++a)
        for (int t = 0; t < 12; ++t)
            if (cnt[a][t] != want[t]) return false;
    return true;
}

// Setup pool (Sec. "Data Collection", App. "Learned Setups"): each side's
// types from entry uniform_below(w0, M) of its pool, mirrored left-right
// when mirroring is on and w1 is odd, (w0, w1) from Philox at counter
// (slot, episode, 0, 7<<24 | side).  Writes G->c.type.
template <int L>
__device__ __noinline__ void pool_types(SmemGame* G, Team<L>, const uint8_t* pool, int M, uint32_t pool_flags,
                                        uint32_t k0, uint32_t k1, uint32_t slot, uint32_t episode)
{
    const Team<L> T;
    for (int p = T.tl; p < kPieces; p += L) {
        const int side = p / 40, i = p - 40 * side;
        const uint4 w = philox(make_uint4(slot, episode, 0u, (7u << 24) | (uint32_t)side), k0, k1);
        const uint32_t e = uniform_below(w.x, (uint32_t)M);
        const bool flip = (pool_flags & ST_POOL_MIRROR) && (w.y & 1u);
        const int row = i / 10, col = i - 10 * row;
        G->c.type[p] = pool[((size_t)side * (size_t)M + e) * 40 + 10 * row + (flip ? 9 - col : col)];
    }
    T.sync();
}

// Restart from a pinned position (App. B.4): its core, board, history ring
// and chase positions, with the slot's new episode number.
template <int L>
__device__ __noinline__ void restart_pinned(SmemGame* G, Team<L>, const RootState* R, uint32_t episode, uint16_t* ring,
                                            uint64_t* pi)
{
    const Team<L> T;
    const uint16_t hrow = G->c.hrow, hcur = G->c.hcur;
    T.sync();
    const uint4* src = reinterpret_cast<const uint4*>(R);
    uint4* dst = reinterpret_cast<uint4*>(G);
    for (int i = T.tl; i < (288 + 112) / 16; i += L) dst[i] = src[i];
    const uint4* rs = reinterpret_cast<const uint4*>(R->ring);
    uint4* rd = reinterpret_cast<uint4*>(ring);
    for (int i = T.tl; i < kRing * 2 / 16; i += L) rd[i] = rs[i];
    const int npi = R->c.n_pi;
    for (int i = T.tl; i < 2 * npi; i += L) pi[i] = R->pi[i];
    T.sync();
    if (T.leader()) {
        G->c.episode = episode;
        G->c.terminated = 0;
        G->c.hrow = hrow;
        G->c.hcur = hcur;
    }
    T.sync();
    derive_state(G, ring, pi, T);
}

// A new game of slot `slot` at `episode`: its pinned position, else the
// setup pool, else the Philox setup.
template <int L>
__device__ __forceinline__ void new_game(SmemGame* G, const Team<L>& T, const ResetSrc& src, uint32_t k0, uint32_t k1,
                                         uint32_t slot, uint32_t episode, uint16_t* ring, uint64_t* pi)
{
    const int pin = src.pin_of ? src.pin_of[slot] : -1;
    if (pin >= 0) {
        restart_pinned(G, T, src.pins + pin, episode, ring, pi);
    } else {
        if (src.pool) pool_types(G, T, src.pool, src.pool_m, src.pool_flags, k0, k1, slot, episode);
        reset_game(G, T, k0, k1, slot, episode, src.pool ? G->c.type : (const uint8_t*)nullptr);
    }
    if (T.leader()) G->c.fresh = kFreshNew;
    T.sync();
}

// Auto-reset inside a launch: the new game, then the moves of its player to
// move (recorded, their mask in mdst when given; their count returned).  One
// out-of-line call on the rare path.
template <int L, bool kRows>
__device__ __noinline__ int restart_slot(SmemGame* G, Team<L>, ResetSrc src, uint32_t k0, uint32_t k1,
                                         uint32_t rule_flags, uint32_t slot, uint32_t episode, uint16_t* ring,
                                         uint64_t* pi, uint32_t* mdst)
{
    const Team<L> T;
    new_game(G, T, src, k0, k1, slot, episode, ring, pi);
    return gen_moves<L, kRows>(G, T, G->c.ply & 1, rule_flags, false, true, pi, mdst);
}

// One ply of slot `slot` (App. B.1): the moves of the player to move are
// recorded in G (sq_cnt, and desc or, with kRows, the mask rows in mdst), n
// of them.  given: the supplied action or -1 for the random policy.  mdst:
// the row that receives the mask of the player to move after the ply (of the
// new game after an auto-reset; all zero for a finished game), or null
// (required with kRows).  staged: a bulk copy may still be reading mdst (the
// team's staging buffer), so it is waited for before mdst is written.  An
// illegal supplied action changes nothing and leaves mdst untouched.
template <int L, bool kRows = false>
__device__ __forceinline__ PlyResult env_ply(SmemGame* G, const Team<L>& T, int& n, const EnvArgs& A, uint32_t slot,
                                             int given, uint16_t* ring, uint64_t* pi, bool& illegal, uint32_t* mdst,
                                             bool staged = false)
{
    PlyResult res;
    // the ply index is read by the leader alone, which is the lane that
    // writes it and the only one whose result is used
    res.action = -1; res.code = 0; res.winner = -1; res.ply_idx = T.leader() ? G->c.ply : 0;
    illegal = false;
    if (G->c.terminated) {
        if (staged) mask_free(T);
        zero_row(mdst, T);
        T.sync();
        return res;
    }
    if (n == 0) {
        if (staged) mask_free(T);
        start_end(G, T, A.R, pi, res.code, res.winner);
    } else {
        int a = given;
        if (a >= 0) {
            const bool ok = kRows ? (a < 10000 && ((rows_of(G)[a >> 5] >> (a & 31)) & 1u))
                                  : move_recorded(G, a, pi, A.R.flags);
            if (!ok) {
                illegal = true;
                T.sync();   // every lane has read the records before the caller rewrites them
                return res;
            }
        } else {
            const uint4 w = philox(make_uint4(slot, G->c.episode, (uint32_t)G->c.ply, 2u << 24), A.k0, A.k1);
            a = select_action<L, kRows>(G, T, uniform_below(w.x, (uint32_t)n), pi, A.R.flags);
        }
        apply_move(G, T, a, ring, pi);
        res.action = a;
        if (staged) mask_free(T);
        check_end<L, kRows>(G, T, A.R, pi, res.code, res.winner, n, mdst);
    }
    if (res.code) {
        if (A.R.flags & kAutoreset) {
            n = restart_slot<L, kRows>(G, T, A.reset, A.k0, A.k1, A.R.flags, slot, G->c.episode + 1, ring, pi, mdst);
        } else {
            if (T.leader()) G->c.terminated = (uint8_t)res.code;
            zero_row(mdst, T);
            n = 0;
            T.sync();   // every lane sees the game as finished before the next ply reads the record
        }
    }
    // (apply_move, gen_moves and a restart end with a team barrier: the
    // record the next ply reads is the same for every lane)
    return res;
}

__device__ __forceinline__ int reward_of(const PlyResult& r)
{
    if (r.code == 1 || r.code == 2) return r.winner == 0 ? 1 : -1;
    return 0;
}

// Per-slot counters: games ended by code 1-5, plies played, red wins, blue wins.
__device__ __forceinline__ void count_result(uint32_t* st, const PlyResult& r)
{
    st[5] += r.action >= 0;
    if (r.code) {
        st[r.code - 1] += 1;
        const int rw = reward_of(r);
        if (rw > 0) st[6] += 1;
        else if (rw < 0) st[7] += 1;
    }
}

template <int L>
__device__ __forceinline__ SmemGame* team_game(unsigned char* smem) { return reinterpret_cast<SmemGame*>(smem) + threadIdx.x / L; }

__global__ void k_env_reset(EnvArgs A, const uint8_t* setups, const uint8_t* which, int first)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const Team<32> T;
    SmemGame* G = team_game<32>(smem);
    const int g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (g >= A.N) return;
    if (which && !which[g]) return;
    const uint8_t* setup = setups ? setups + 80 * (size_t)g : nullptr;
    if (setup && !setup_counts_ok(setup)) {
        if (T.leader()) latch(A.status, ST_ERR_BAD_POSITION, g);
        return;
    }
    uint32_t episode = 0;
    if (!first) {
        load_core(G, A.core + g, T);
        episode = G->c.episode + 1;
    }
    if (first && T.tl < 8) A.stats[8 * (size_t)g + T.tl] = 0;
    uint16_t* ring = A.ring + (size_t)g * kRing;
    uint64_t* pi = A.pi + (size_t)g * kPiWords;
    if (setup) {
        reset_game(G, T, A.k0, A.k1, (uint32_t)g, episode, setup);
        if (T.leader()) G->c.fresh = kFreshSetup;
    } else {
        new_game(G, T, A.reset, A.k0, A.k1, (uint32_t)g, episode, ring, pi);
    }
    const int n = gen_moves(G, T, G->c.ply & 1, A.R.flags, false, false, pi, (uint32_t*)nullptr);
    if (T.leader()) G->c.n_legal = (uint16_t)n;
    store_core(G, A.core + g, T);
}

// History ring (App. B.1: a circular buffer of past steps): the row of a
// step holds, per slot, the action played (bits 0-13, 0x3FFF for none), how
// the game began if the step's state was its first (bits 14-15, kFresh*),
// the ending code reported by the step (bits 16-18) and red's reward + 1
// (bits 19-20).  The leader notes the mark before the ply (the ply may start
// the next game) ...
template <int L>
__device__ __forceinline__ void hist_before(SmemGame* G, const Team<L>& T)
{
    if (T.leader()) {
        G->c.hcur = G->c.fresh;
        G->c.fresh = 0;
    }
}

// ... and writes the row after it.
__device__ __forceinline__ void hist_after(SmemGame* G, const EnvArgs& A, int g, const PlyResult& r)
{
    const uint32_t v = (r.action >= 0 ? (uint32_t)r.action : 0x3FFFu) | ((uint32_t)G->c.hcur << 14) |
                       ((uint32_t)r.code << 16) | ((uint32_t)(reward_of(r) + 1) << 19);
    A.hist[(size_t)G->c.hrow * (size_t)A.N + (size_t)g] = v;
    G->c.hrow = (uint16_t)(G->c.hrow + 1 == A.H ? 0 : G->c.hrow + 1);
}

template <int L>
__global__ void __launch_bounds__(128, 6) k_env_step(EnvArgs A, const int16_t* actions, int16_t* action_out, int8_t* reward_out,
                           uint8_t* done_out, int16_t* ply_out, uint8_t* mask_out)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const Team<L> T;
    SmemGame* G = team_game<L>(smem);
    const int g = blockIdx.x * (blockDim.x / L) + threadIdx.x / L;
    if (g >= A.N) return;
    uint16_t* ring = A.ring + (size_t)g * kRing;
    uint64_t* pi = A.pi + (size_t)g * kPiWords;
    load_core(G, A.core + g, T);
    build_board(G, T);
    derive_state(G, ring, pi, T);
    const int P = G->c.ply & 1;
    int n = 0;
    if (!G->c.terminated) n = gen_moves(G, T, P, A.R.flags, false, true, pi, (uint32_t*)nullptr);
    bool illegal = false;
    const int given = actions ? (int)actions[g] : -1;
    if (A.hist) {
        if (T.leader()) G->c.hrow = (uint16_t)(*A.now % A.H);
        hist_before(G, T);
    }
    uint32_t* mdst = mask_out ? reinterpret_cast<uint32_t*>(mask_out + (size_t)g * kMaskBytes) : nullptr;
    const PlyResult r = env_ply(G, T, n, A, (uint32_t)g, given, ring, pi, illegal, mdst);
    // an illegal action changed nothing: the mask is the one of the player still to move
    if (illegal && mdst) gen_moves(G, T, P, A.R.flags, false, true, pi, mdst);
    if (T.leader()) {
        if (A.hist) hist_after(G, A, g, r);
        if (illegal) latch(A.status, ST_ERR_ILLEGAL_ACTION, g);
        if (action_out) action_out[g] = (int16_t)r.action;
        if (reward_out) reward_out[g] = (int8_t)reward_of(r);
        if (done_out) done_out[g] = (uint8_t)r.code;
        if (ply_out) ply_out[g] = (int16_t)r.ply_idx;
        if (!illegal) {
            uint32_t st[8];
            uint32_t* gs = A.stats + 8 * (size_t)g;
#pragma unroll
            for (int k = 0; k < 8; ++k) st[k] = gs[k];
            count_result(st, r);
#pragma unroll
            for (int k = 0; k < 8; ++k) gs[k] = st[k];
        }
        G->c.n_legal = (uint16_t)n;
    }
    store_core(G, A.core + g, T);   // an illegal action changed nothing but the history marks
}

// Persistent form: each team claims gpf work units at a time from a global
// counter, a unit being one part of a slot's n_steps plies (nsplit parts,
// all first parts before any second part, and so on), and plays it keeping
// the game in shared memory.  Splitting the plies fills the last wave of
// units when the slots are a little more than a whole number of resident
// games (65,536 slots over 14,592 games: 4.49 waves of whole slots, 8.98
// of halves).  A part waits for its slot's previous part, which was claimed
// a wave or more earlier and has normally finished; the wait is bounded
// and latches ST_ERR_TIMEOUT for the slot if it ever ran out.
constexpr int kMinPartPlies = 256;      // no part shorter than this many plies
constexpr int kMaxParts = 4;
constexpr int kMaxSplitPlies = 32768;   // launches longer than this are not split (a part's wait stays short)
#ifndef ST_PART_SPIN_LIMIT
#define ST_PART_SPIN_LIMIT (1ll << 22)   // polls of ~0.3-1 us: a few seconds
#endif
constexpr long long kPartSpinLimit = ST_PART_SPIN_LIMIT;
// A work unit's start: the slot's game into the team's record (core,
// board, derived state), the staging buffer free of the previous unit's
// last copy, the moves of the player to move recorded, the launch counters
// cleared.  Returns the number of legal moves.  Out of line, like the other
// per-unit steps, so that the step loop's registers are allocated alone.
template <int L>
__device__ __noinline__ int unit_start(SmemGame* G, const GameCore* core, uint16_t* ring, uint64_t* pi,
                                       uint32_t rule_flags, bool staged, Team<L>)
{
    const Team<L> T;
    load_core(G, core, T);
    build_board(G, T);
    derive_state(G, ring, pi, T);
    if (staged) mask_free(T);   // the previous unit's last copy has read the staging buffer
    int n = 0;
    if (!G->c.terminated) n = gen_moves<L, true>(G, T, G->c.ply & 1, rule_flags, false, true, pi, rows_of(G));
    // the launch's counters live in shared memory, not in registers that
    // every engine call would have to save
    for (int k = T.tl; k < 8; k += L) G->stat[k] = 0;
    return n;
}

// A work unit's end: the launch counters added to the slot's, the record
// back to the slot's core; with done (the slot's count of finished parts),
// the release of the slot's next part: the record, counters, history ring
// and chase store are in global memory first.
template <int L>
__device__ __noinline__ void unit_finish(SmemGame* G, GameCore* core, uint32_t* stats, int n, int32_t* done, Team<L>)
{
    const Team<L> T;
    if (T.leader()) {
#pragma unroll
        for (int k = 0; k < 8; ++k) stats[k] += G->stat[k];
        G->c.n_legal = (uint16_t)n;
    }
    store_core(G, core, T);
    if (done) {
        __threadfence();
        T.sync();
        if (T.leader()) atomicAdd(done, 1);   // parts end in order: the count of parts done
    }
}

// Has the slot's part h-1 been stored (its count of finished parts, *done,
// reached h; the release is unit_finish's)?  The team's first lane polls,
// bounded, then fences; team-uniform result.  Out of line: the wait's
// registers stay out of the step loop's allocation.
template <int L>
__device__ __noinline__ bool part_ready(int32_t* done, int h, Team<L>)
{
    const Team<L> T;
    int ok = 1;
    if (T.leader()) {
        long long spins = 0;
        while (atomicAdd(done, 0) < h && spins < kPartSpinLimit) {
            __nanosleep(256);
            ++spins;
        }
        ok = spins < kPartSpinLimit;
        __threadfence();
    }
    return T.shfl(ok, 0) != 0;
}

// At most 256 threads per block and 3 blocks per SM: <= 85 (80) registers a
// thread; shared memory, not registers, bounds the resident teams.
constexpr int kRunMaxWarps = 8;
template <int L, bool kHist>
__global__ void __launch_bounds__(32 * kRunMaxWarps, 3) k_env_run(EnvArgs A, int32_t* queue, int n_steps, int ring_steps, int gpf,
                                                 int16_t* action_ring, int8_t* reward_ring, uint8_t* done_ring,
                                                 int16_t* ply_ring, uint8_t* mask_ring, int nsplit,
                                                 int part, int32_t* part_done)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const Team<L> T;
    // the team's game record in row mode: no descriptors, the mask of the
    // player to move right after it (rows_of), which is also the buffer the
    // bulk copies send to the ring
    SmemGame* G = reinterpret_cast<SmemGame*>(smem + (size_t)(threadIdx.x / L) * kRowsRecordBytes);
    // (part = ceil(n_steps / nsplit) plies, a launch parameter: like every
    // per-launch bound, it is read from the parameter bank rather than held
    // in a register across the plies)
    for (;;) {
        const int units = A.N * nsplit;
        // each team claims its own units: no collective spans more than one team
        int first = 0;
        if (T.leader()) first = atomicAdd(queue, gpf);
        first = T.shfl(first, 0);
        if (first >= units) break;
        for (int gi = 0; gi < gpf; ++gi) {
            const int u = first + gi;
            if (u >= A.N * nsplit) break;
            const int h = u / A.N, g = u - h * A.N;          // part h of slot g
            const int j0 = h * part, j1 = min(n_steps, j0 + part);
            if (h > 0 && !part_ready(part_done + g, h, T)) {
                if (T.leader()) latch(A.status, ST_ERR_TIMEOUT, g);
                continue;
            }
            uint16_t* ring = A.ring + (size_t)g * kRing;
            uint64_t* pi = A.pi + (size_t)g * kPiWords;
            int n = unit_start<L>(G, A.core + g, ring, pi, A.R.flags, mask_ring != nullptr, T);
            if (kHist && T.leader()) G->c.hrow = (uint16_t)((*A.now + j0) % A.H);
            int row = j0 % ring_steps;   // output ring row of ply j: j mod ring_steps
            // a countdown, so that neither the part's bounds nor its index
            // stay live in registers across the plies
            for (int left = j1 - j0; left > 0; --left) {
                bool illegal;
                if (kHist) hist_before(G, T);
                const size_t o = (size_t)row * (size_t)A.N + (size_t)g;
                if (++row == ring_steps) row = 0;
                // the mask of the player to move after the ply is rendered into
                // the staging buffer, which the next ply's selection reads, and
                // leaves it by a bulk copy
                const PlyResult r = env_ply<L, true>(G, T, n, A, (uint32_t)g, -1, ring, pi, illegal, rows_of(G),
                                                     mask_ring != nullptr);
                if (T.leader()) {
                    if (kHist) hist_after(G, A, g, r);
                    count_result(G->stat, r);
                    if (action_ring) action_ring[o] = (int16_t)r.action;
                    if (reward_ring) reward_ring[o] = (int8_t)reward_of(r);
                    if (done_ring) done_ring[o] = (uint8_t)r.code;
                    if (ply_ring) ply_ring[o] = (int16_t)r.ply_idx;
                }
                if (mask_ring) write_mask_async(rows_of(G), T, mask_ring + o * kMaskBytes);
            }
            unit_finish<L>(G, A.core + g, A.stats + 8 * (size_t)g, n, nsplit > 1 ? part_done + g : nullptr, T);
        }
    }
    // the team's last mask copies have landed before it leaves
    if (mask_ring && T.leader()) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Warp per slot: the random policy's action at the current state (the
// action the next step would play with actions NULL), -1 for an ended game
// or a player without a legal move (App. B.1 SampleRandomLegalAction).
__global__ void k_env_sample(EnvArgs A, int16_t* out)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const Team<32> T;
    SmemGame* G = team_game<32>(smem);
    const int g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (g >= A.N) return;
    uint16_t* ring = A.ring + (size_t)g * kRing;
    uint64_t* pi = A.pi + (size_t)g * kPiWords;
    load_core(G, A.core + g, T);
    build_board(G, T);
    derive_state(G, ring, pi, T);
    int a = -1;
    if (!G->c.terminated) {
        const int n = gen_moves(G, T, G->c.ply & 1, A.R.flags, false, true, pi, (uint32_t*)nullptr);
        if (n > 0) {
            const uint4 w = philox(make_uint4((uint32_t)g, G->c.episode, (uint32_t)G->c.ply, 2u << 24), A.k0, A.k1);
            a = select_action(G, T, uniform_below(w.x, (uint32_t)n), pi, A.R.flags);
        }
    }
    if (T.leader()) out[g] = (int16_t)a;
}

// ----------------------------------------------------------------- snapshots

// Team: the snapshot of game G (history ring `ring`) into o.
template <int L>
__device__ void export_position(const SmemGame* G, const uint16_t* ring, st_position* o, const Team<L>& T)
{
    uint8_t* ob = reinterpret_cast<uint8_t*>(o);
    const int lane = T.tl;
    for (int b = lane; b < 240; b += L) ob[b] = reinterpret_cast<const uint8_t*>(&G->c)[b];
    for (int h = lane; h < 256; h += L) o->hist[h] = (uint16_t)hist_at(G, ring, h);
    if (lane == 0) {
        o->ply = G->c.ply;
        o->battleless = G->c.battleless;
        o->last_battle = G->c.last_battle;
        o->chaser = G->c.chaser;
        o->chase_plies = G->c.chase_plies;
        o->reserved0 = 0;
        for (int p = 0; p < 2; ++p) {
            o->ts_pid[p] = G->c.ts_pid[p];
            o->ts_len[p] = G->c.ts_len[p];
            for (int k = 0; k < 4; ++k) o->ts_sq[p][k] = k < G->c.ts_len[p] ? G->c.ts_sq[p][k] : kNone;
        }
        for (int k = 0; k < 12; ++k) o->reserved1[k] = 0;
    }
    T.sync();
}

__global__ void k_env_export(EnvArgs A, const int32_t* idx, int n, st_position* out)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const Team<32> T;
    SmemGame* G = team_game<32>(smem);
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= n) return;
    const int g = idx[i];
    if (g < 0 || g >= A.N) {
        if (T.leader()) latch(A.status, ST_ERR_BAD_POSITION, i);
        return;
    }
    load_core(G, A.core + g, T);
    export_position(G, A.ring + (size_t)g * kRing, out + i, T);
}

__global__ void k_env_import(EnvArgs A, const int32_t* idx, int n, const st_position* in)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const Team<32> T;
    SmemGame* G = team_game<32>(smem);
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= n) return;
    const int g = idx[i];
    if (g < 0 || g >= A.N) {
        if (T.leader()) latch(A.status, ST_ERR_BAD_POSITION, i);
        return;
    }
    // keep the episode counter of the slot
    const uint32_t episode = A.core[g].episode;
    uint16_t* ring = A.ring + (size_t)g * kRing;
    uint64_t* pi = A.pi + (size_t)g * kPiWords;
    const int bad = import_position(G, in + i, ring, pi);
    if (bad) {
        if (T.leader()) latch(A.status, ST_ERR_BAD_POSITION, g);
        return;
    }
    const int nl = gen_moves(G, T, G->c.ply & 1, A.R.flags, false, false, pi, (uint32_t*)nullptr);
    if (T.leader()) {
        G->c.episode = episode;
        G->c.n_legal = (uint16_t)nl;
        G->c.fresh = kFreshImport;
    }
    store_core(G, A.core + g, T);
}

// Warp per entry: the pinned record of states[i] for slot idx[i] (the later
// entry wins for a slot listed twice).
__global__ void k_env_pin(EnvArgs A, const int32_t* idx, int n, const st_position* states, RootState* recs,
                          int32_t* pin_of)
{
    extern __shared__ __align__(16) unsigned char smem[];
    RolloutSmem* S = reinterpret_cast<RolloutSmem*>(smem) + (threadIdx.x >> 5);
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= n) return;
    const int lane = threadIdx.x & 31;
    const int g = idx[i];
    if (g < 0 || g >= A.N) {
        if (lane == 0) latch(A.status, ST_ERR_BAD_POSITION, i);
        return;
    }
    const int bad = build_root(S, states + i, recs + i);
    if (lane == 0) {
        if (bad) latch(A.status, ST_ERR_BAD_POSITION, i);
        else atomicMax(&pin_of[g], i);
    }
}

// ----------------------------------------------------------------- history queries
// Queries about the state at step t (App. B.1 historical queries): the game
// holding a slot at step t is rebuilt from its start (the latest row in the
// window with a start mark) by replaying the recorded actions.
struct HistQuery {
    const uint32_t* hist;
    int H;
    long long now;    // steps taken
    long long lo;     // first step whose row is in the window
    long long floor;  // games begun before this step used other reset sources
    long long t;
};

__device__ __forceinline__ uint32_t hist_row(const HistQuery& Q, int N, int g, long long s)
{
    return Q.hist[(size_t)(s % Q.H) * (size_t)N + (size_t)g];
}

__device__ __forceinline__ uint32_t row_mark(uint32_t v) { return (v >> 14) & 3u; }
__device__ __forceinline__ uint32_t row_done(uint32_t v) { return (v >> 16) & 7u; }

// Team: the latest step s in [lo, hi] whose row has a nonzero field
// (field(v) != 0), -1 if none; val: that field.
template <int L, typename F>
__device__ long long latest_row(const HistQuery& Q, int N, int g, long long hi, F field, uint32_t& val,
                                const Team<L>& T)
{
    for (long long base = hi; base >= Q.lo; base -= L) {
        const long long s = base - T.tl;
        const uint32_t f = s >= Q.lo ? field(hist_row(Q, N, g, s)) : 0u;
        const uint32_t m = T.ballot(f != 0);
        if (m) {
            const int l = __ffs(m) - 1;
            val = (uint32_t)T.shfl((int)f, l);
            return base - l;
        }
    }
    val = 0;
    return -1;
}

// Team: where the game holding slot g at step Q.t began (-1: before the
// window) and how (kFresh*).  At t = now a pending mark of the slot counts.
template <int L>
__device__ long long game_start(const HistQuery& Q, const GameCore* cur, int N, int g, int& kind, const Team<L>& T)
{
    if (Q.t == Q.now && cur->fresh) {
        kind = cur->fresh;
        return Q.now;
    }
    uint32_t k = 0;
    const long long s0 = latest_row(Q, N, g, Q.t == Q.now ? Q.now - 1 : Q.t,
                                    [](uint32_t v) { return row_mark(v); }, k, T);
    kind = (int)k;
    return s0;
}

// Team: the episode number of the game that began at step s0 (counted back
// from the slot's current episode over the later new games and resets).
template <int L>
__device__ uint32_t episode_at(const HistQuery& Q, const GameCore* cur, int N, int g, long long s0, const Team<L>& T)
{
    int cnt = 0;
    for (long long s = s0 + 1 + T.tl; s < Q.now; s += L) {
        const uint32_t m = row_mark(hist_row(Q, N, g, s));
        cnt += (m == kFreshNew || m == kFreshSetup);
    }
    cnt = T.sum(cnt);
    const int pending = (s0 < Q.now && (cur->fresh == kFreshNew || cur->fresh == kFreshSetup)) ? 1 : 0;
    return cur->episode - (uint32_t)cnt - (uint32_t)pending;
}

// A team's record for rebuilding a past position: the game and its history
// ring; its chase store is the team's slot of a global scratch array.
struct __align__(16) HistSmem {
    SmemGame g;
    uint16_t ring[kRing];
};

// Team of L lanes per slot: the position at step t, how the game stood
// (ended: its ending code if it was over, since: steps since the step that
// ended it), and a status (0 ok; 2 the game began before the window or
// before the last change of reset sources; 3 it began from given setups or
// an import; the current step always has its position).  The rebuild replays
// the game's recorded moves from its start, the team's first lane playing
// them; with several teams per warp, several slots replay side by side.
// pi_scratch: kPiWords words per slot.
template <int L>
__global__ void k_env_hist_positions(EnvArgs A, HistQuery Q, st_position* out, uint8_t* status, uint8_t* ended,
                                     int32_t* since, uint64_t* pi_scratch)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const Team<L> T;
    const int team = threadIdx.x / L;
    HistSmem* S = reinterpret_cast<HistSmem*>(smem) + team;
    const int g = blockIdx.x * (blockDim.x / L) + team;
    if (g >= A.N) return;   // a whole team leaves; collectives are per team
    uint64_t* pi = pi_scratch + (size_t)g * kPiWords;
    const GameCore* cur = A.core + g;
    int kind = 0;
    const long long s0 = game_start(Q, cur, A.N, g, kind, T);
    // the step that ended the game, if it is over
    uint32_t code = 0;
    long long e = -1;
    if (Q.t > Q.lo) {
        const long long from = s0 >= 0 ? s0 : Q.lo;
        HistQuery Qe = Q;
        Qe.lo = from;
        if (Q.t - 1 >= from) e = latest_row(Qe, A.N, g, Q.t - 1, [](uint32_t v) { return row_done(v); }, code, T);
    }
    if (Q.t == Q.now && cur->terminated && e < 0) code = cur->terminated;
    if (T.leader()) {
        if (ended) ended[g] = (uint8_t)code;
        if (since) since[g] = e >= 0 ? (int32_t)(Q.t - e) : (code ? -1 : 0);
    }
    uint8_t st = 0;
    if (Q.t == Q.now) {
        load_core(&S->g, cur, T);
        export_position(&S->g, A.ring + (size_t)g * kRing, out + g, T);
    } else if (s0 < 0 || s0 < Q.floor) {
        st = 2;
    } else if (kind != kFreshNew) {
        st = 3;
    } else {
        const uint32_t ep = episode_at(Q, cur, A.N, g, s0, T);
        new_game(&S->g, T, A.reset, A.k0, A.k1, (uint32_t)g, ep, S->ring, pi);
        for (long long base = s0; base < Q.t; base += L) {
            const long long s = base + T.tl;
            const uint32_t v = s < Q.t ? hist_row(Q, A.N, g, s) : 0x3FFFu;
            const int cnt = (int)min((long long)L, Q.t - base);
            for (int j = 0; j < cnt; ++j) {
                const int a = T.shfl((int)v, j) & 0x3FFF;
                if (a != 0x3FFF) apply_move(&S->g, T, a, S->ring, pi);
            }
        }
        export_position(&S->g, S->ring, out + g, T);
    }
    if (T.leader() && status) status[g] = st;
}

// Thread per slot: the row of step t (t < now): action (-1 none), ending
// code, red's reward, start mark.
__global__ void k_env_hist_steps(int N, HistQuery Q, int16_t* action, uint8_t* done, int8_t* reward, uint8_t* start)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= N) return;
    const uint32_t v = hist_row(Q, N, g, Q.t);
    const uint32_t a = v & 0x3FFFu;
    if (action) action[g] = a == 0x3FFFu ? (int16_t)-1 : (int16_t)a;
    if (done) done[g] = (uint8_t)row_done(v);
    if (reward) reward[g] = (int8_t)((int)((v >> 19) & 3u) - 1);
    if (start) start[g] = (uint8_t)row_mark(v);
}

// Warp per slot: the setup and the action log of the game at step t, for
// st_obs_encode (status 0 ok, 2 and 3 as for positions, 4 a pinned start,
// 5 more than L actions).
__global__ void k_env_hist_logs(EnvArgs A, HistQuery Q, int L, uint8_t* setups, int16_t* logs, int16_t* plies,
                                uint8_t* status)
{
    extern __shared__ __align__(16) unsigned char smem[];
    SmemGame* G = team_game<32>(smem);
    const int g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (g >= A.N) return;
    const Team<32> T;
    const int lane = T.tl;
    const GameCore* cur = A.core + g;
    int kind = 0;
    const long long s0 = game_start(Q, cur, A.N, g, kind, T);
    int16_t* log = logs + (size_t)g * (size_t)L;
    uint8_t st = 0;
    if (s0 < 0 || s0 < Q.floor) st = 2;
    else if (kind != kFreshNew) st = 3;
    else if (A.reset.pin_of && A.reset.pin_of[g] >= 0) st = 4;
    int n = 0;
    if (!st) {
        const uint32_t ep = episode_at(Q, cur, A.N, g, s0, T);
        if (A.reset.pool) pool_types(G, T, A.reset.pool, A.reset.pool_m, A.reset.pool_flags, A.k0, A.k1, (uint32_t)g, ep);
        reset_game(G, T, A.k0, A.k1, (uint32_t)g, ep, A.reset.pool ? G->c.type : (const uint8_t*)nullptr);
        for (int i = lane; i < kPieces; i += 32) setups[(size_t)g * kPieces + i] = G->c.type[i];
        for (long long base = s0; base < Q.t; base += 32) {
            const long long s = base + lane;
            const uint32_t a = s < Q.t ? (hist_row(Q, A.N, g, s) & 0x3FFFu) : 0x3FFFu;
            const bool has = a != 0x3FFFu;
            const uint32_t m = __ballot_sync(~0u, has);
            const int o = n + __popc(m & ((1u << lane) - 1u));
            if (has && o < L) log[o] = (int16_t)a;
            n += __popc(m);
        }
        if (n > L) st = 5;
    } else {
        for (int i = lane; i < kPieces; i += 32) setups[(size_t)g * kPieces + i] = 0;
    }
    for (int i = n + lane; i < L; i += 32) log[i] = -1;
    if (lane == 0) {
        plies[g] = (int16_t)(st ? 0 : n);
        if (status) status[g] = st;
    }
}

__global__ void k_env_advance(long long* now, int n)
{
    *now += n;
}

__global__ void k_env_clear_marks(GameCore* core, int N)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < N) core[g].fresh = 0;
}

EnvArgs env_args(st_env* e)
{
    EnvArgs a;
    a.core = e->core; a.ring = e->ring; a.pi = e->pi; a.stats = e->stats; a.status = e->status;
    a.N = e->N; a.k0 = (uint32_t)e->seed; a.k1 = (uint32_t)(e->seed >> 32); a.R = e->rules;
    a.reset.pool = e->pool; a.reset.pool_m = e->pool_m; a.reset.pool_flags = e->pool_flags;
    a.reset.pin_of = e->n_pins > 0 ? e->pin_of : nullptr;
    a.reset.pins = e->pins;
    a.hist = e->hist;
    a.H = e->H;
    a.now = e->d_now;
    return a;
}

HistQuery hist_query(st_env* e, long long t)
{
    HistQuery q;
    q.hist = e->hist;
    q.H = e->H;
    q.now = e->now;
    q.lo = std::max(e->hist_start, e->now - (long long)e->H);
    q.floor = e->cfg_floor;
    q.t = t;
    return q;
}

constexpr int kPlainWarps = 4;

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) { cudaGetDevice(&prev); if (prev != dev) cudaSetDevice(dev); }
    ~DeviceGuard() { int cur; cudaGetDevice(&cur); if (prev >= 0 && cur != prev) cudaSetDevice(prev); }
};

// Dynamic shared memory of one block of the persistent launch.
size_t run_smem(int wpb, int gpw) { return (size_t)wpb * gpw * kRowsRecordBytes; }

template <int L>
cudaError_t run_occupancy_t(int wpb, int* occ)
{
    const size_t smem = run_smem(wpb, 32 / L);
    // both forms of the kernel (with and without the history ring) get the
    // shared-memory limit; their occupancy is that of the form without it
    cudaError_t e = cudaFuncSetAttribute(k_env_run<L, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_env_run<L, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_env_run<L, false>, 32 * wpb, smem);
    if (e != cudaSuccess) cudaGetLastError();   // leave no pending error behind for later launches
    return e;
}

cudaError_t run_occupancy(int wpb, int gpw, int* occ)
{
    switch (gpw) {
    case 8: return run_occupancy_t<4>(wpb, occ);
    case 4: return run_occupancy_t<8>(wpb, occ);
    case 2: return run_occupancy_t<16>(wpb, occ);
    default: return run_occupancy_t<32>(wpb, occ);
    }
}

// Parts per slot of a persistent launch over N slots by R resident games:
// only when the slots outnumber the resident games (more than one wave, so
// each part is claimed a wave after the slot's previous part), for launches
// of at most kMaxSplitPlies plies (a part waits at most about one part's
// time) and parts of at least kMinPartPlies plies; the count whose last
// wave is fullest (the launch lasts about ceil(n N / R) / n whole-slot
// waves), the fewest parts within 2% of the best.
int parts_per_slot(int N, int R, int n_steps)
{
    if (R <= 0 || N <= R || n_steps > kMaxSplitPlies) return 1;
    const double w = (double)N / (double)R;
    double best = 1e30;
    for (int n = 1; n <= kMaxParts && n_steps >= n * kMinPartPlies; ++n)
        best = std::min(best, std::ceil(n * w) / n);
    for (int n = 1; n <= kMaxParts && n_steps >= n * kMinPartPlies; ++n)
        if (std::ceil(n * w) / n <= 1.02 * best) return n;
    return 1;
}

template <int L>
void launch_run_t(st_env* e, const EnvArgs& a, int blocks, int n_steps, int ring_steps, int16_t* action_ring,
                  int8_t* reward_ring, uint8_t* done_ring, int16_t* ply_ring, uint8_t* mask_ring, int nsplit)
{
    if (a.hist)
        k_env_run<L, true><<<blocks, 32 * e->wpb, run_smem(e->wpb, 32 / L), e->stream>>>(
            a, e->queue, n_steps, ring_steps, e->gpf, action_ring, reward_ring, done_ring, ply_ring, mask_ring, nsplit,
            (n_steps + nsplit - 1) / nsplit, e->part_done);
    else
        k_env_run<L, false><<<blocks, 32 * e->wpb, run_smem(e->wpb, 32 / L), e->stream>>>(
            a, e->queue, n_steps, ring_steps, e->gpf, action_ring, reward_ring, done_ring, ply_ring, mask_ring, nsplit,
            (n_steps + nsplit - 1) / nsplit, e->part_done);
}

void launch_run(st_env* e, const EnvArgs& a, int blocks, int n_steps, int ring_steps, int16_t* action_ring,
                int8_t* reward_ring, uint8_t* done_ring, int16_t* ply_ring, uint8_t* mask_ring, int nsplit)
{
    switch (e->gpw) {
    case 8: launch_run_t<4>(e, a, blocks, n_steps, ring_steps, action_ring, reward_ring, done_ring, ply_ring, mask_ring, nsplit); break;
    case 4: launch_run_t<8>(e, a, blocks, n_steps, ring_steps, action_ring, reward_ring, done_ring, ply_ring, mask_ring, nsplit); break;
    case 2: launch_run_t<16>(e, a, blocks, n_steps, ring_steps, action_ring, reward_ring, done_ring, ply_ring, mask_ring, nsplit); break;
    default: launch_run_t<32>(e, a, blocks, n_steps, ring_steps, action_ring, reward_ring, done_ring, ply_ring, mask_ring, nsplit);
    }
}

}  // namespace

extern "C" st_status st_env_create(const st_env_config* cfg, st_env** out)
{
    ST_NVTX("st_env_create");
    ST_CHECK_ARG(cfg && out, "st_env_create: null argument");
    ST_CHECK_ARG(cfg->num_games >= 1 && cfg->num_games <= ST_MAX_GAMES, "st_env_create: num_games %d out of range",
                 cfg->num_games);
    ST_CHECK_ARG(rules_ok(&cfg->rules), "st_env_create: invalid rules");
    ST_CHECK_ARG((cfg->env_flags & ~ST_AUTORESET) == 0, "st_env_create: unknown env_flags");
    int ndev = 0;
    ST_CUDA(cudaGetDeviceCount(&ndev));
    ST_CHECK_ARG(cfg->device >= 0 && cfg->device < ndev, "st_env_create: device %d not present", cfg->device);
    *out = nullptr;
    DeviceGuard guard(cfg->device);
    st_env* e = new st_env();
    e->device = cfg->device;
    e->stream = reinterpret_cast<cudaStream_t>(cfg->stream);
    e->N = cfg->num_games;
    e->seed = cfg->seed;
    e->rules.k = cfg->rules.battleless_limit;
    e->rules.cap = cfg->rules.max_plies;
    e->rules.flags = cfg->rules.flags | (cfg->env_flags & ST_AUTORESET ? kAutoreset : 0u);
    const size_t N = (size_t)e->N;
    cudaError_t err = cudaSuccess;
    err = cudaMalloc(&e->core, N * sizeof(GameCore));
    if (err == cudaSuccess) err = cudaMalloc(&e->ring, N * kRing * sizeof(uint16_t));
    if (err == cudaSuccess) err = cudaMalloc(&e->pi, N * kPiWords * sizeof(uint64_t));
    if (err == cudaSuccess) err = cudaMalloc(&e->stats, N * 8 * sizeof(uint32_t));
    if (err == cudaSuccess) err = cudaMalloc(&e->status, 2 * sizeof(int32_t));
    if (err == cudaSuccess) err = cudaMalloc(&e->queue, sizeof(int32_t));
    if (err == cudaSuccess) err = cudaMalloc(&e->part_done, N * sizeof(int32_t));
    if (err != cudaSuccess) {
        stg::set_error("st_env_create: device allocation failed: %s", cudaGetErrorString(err));
        cudaGetLastError();
        st_env_destroy(e);
        return ST_ERR_OOM;
    }
    e->sms = sm_count();
    const int32_t init_status[2] = {0, 0x7FFFFFFF};
    err = cudaMemcpyAsync(e->status, init_status, sizeof(init_status), cudaMemcpyHostToDevice, e->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(e->stream);
    if (err != cudaSuccess) {
        stg::set_error("st_env_create: %s", cudaGetErrorString(err));
        st_env_destroy(e);
        return ST_ERR_CUDA;
    }
    EnvArgs a = env_args(e);
    const int blocks = (e->N + kPlainWarps - 1) / kPlainWarps;
    k_env_reset<<<blocks, 32 * kPlainWarps, kPlainWarps * sizeof(SmemGame), e->stream>>>(a, nullptr, nullptr, 1);
    err = cudaGetLastError();
    if (err == cudaSuccess) err = run_occupancy(e->wpb, e->gpw, &e->max_bps);
    if (err != cudaSuccess) {
        stg::set_error("st_env_create: %s", cudaGetErrorString(err));
        st_env_destroy(e);
        return ST_ERR_CUDA;
    }
    *out = e;
    return ST_OK;
}

extern "C" st_status st_env_destroy(st_env* e)
{
    ST_NVTX("st_env_destroy");
    if (!e) return ST_OK;
    DeviceGuard guard(e->device);
    cudaStreamSynchronize(e->stream);
    if (e->graph) cudaGraphExecDestroy(e->graph);
    cudaFree(e->core); cudaFree(e->ring); cudaFree(e->pi); cudaFree(e->stats);
    cudaFree(e->status); cudaFree(e->queue); cudaFree(e->part_done);
    cudaFree(e->pool); cudaFree(e->pin_of); cudaFree(e->pins);
    cudaFree(e->hist); cudaFree(e->d_now);
    delete e;
    return ST_OK;
}

extern "C" st_status st_env_reset(st_env* e, const uint8_t* setups, const uint8_t* which)
{
    ST_NVTX("st_env_reset");
    ST_CHECK_ARG(e, "st_env_reset: null env");
    DeviceGuard guard(e->device);
    EnvArgs a = env_args(e);
    const int blocks = (e->N + kPlainWarps - 1) / kPlainWarps;
    k_env_reset<<<blocks, 32 * kPlainWarps, kPlainWarps * sizeof(SmemGame), e->stream>>>(a, setups, which, 0);
    ST_CUDA(cudaGetLastError());
    return ST_OK;
}

extern "C" st_status st_env_step(st_env* e, const int16_t* actions, int16_t* action_out, int8_t* reward_out,
                                 uint8_t* done_out, int16_t* ply_out, uint8_t* mask_out)
{
    ST_NVTX("st_env_step");
    ST_CHECK_ARG(e, "st_env_step: null env");
    ST_CHECK_ARG(!mask_out || aligned16(mask_out), "st_env_step: mask_out must be 16-byte aligned");
    DeviceGuard guard(e->device);
    EnvArgs a = env_args(e);
    // teams of kStepLanes lanes: 32 / kStepLanes slots per warp (4 lanes: 8
    // slots; a team size the tuned persistent step does not use, whose
    // out-of-line engine calls it would otherwise share)
    constexpr int kStepLanes = 4, kGames = kPlainWarps * 32 / kStepLanes;
    const int blocks = (e->N + kGames - 1) / kGames;
    k_env_step<kStepLanes><<<blocks, 32 * kPlainWarps, kGames * sizeof(SmemGame), e->stream>>>(
        a, actions, action_out, reward_out, done_out, ply_out, mask_out);
    ST_CUDA(cudaGetLastError());
    if (e->hist) {
        k_env_advance<<<1, 1, 0, e->stream>>>(e->d_now, 1);
        ST_CUDA(cudaGetLastError());
    }
    e->now += 1;
    return ST_OK;
}

extern "C" st_status st_env_set_launch(st_env* e, int32_t warps_per_block, int32_t blocks_per_sm,
                                       int32_t games_per_warp, int32_t games_per_fetch)
{
    ST_NVTX("st_env_set_launch");
    ST_CHECK_ARG(e, "st_env_set_launch: null env");
    ST_CHECK_ARG(warps_per_block >= 1 && warps_per_block <= kRunMaxWarps, "st_env_set_launch: warps_per_block 1..%d",
                 kRunMaxWarps);
    ST_CHECK_ARG(blocks_per_sm >= 0 && blocks_per_sm <= 64, "st_env_set_launch: blocks_per_sm 0..64");
    ST_CHECK_ARG(games_per_warp == 1 || games_per_warp == 2 || games_per_warp == 4 || games_per_warp == 8,
                 "st_env_set_launch: games_per_warp 1, 2, 4 or 8");
    ST_CHECK_ARG(games_per_fetch >= 1 && games_per_fetch <= 4096, "st_env_set_launch: games_per_fetch 1..4096");
    DeviceGuard guard(e->device);
    int smem_max = 0;
    ST_CUDA(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, e->device));
    ST_CHECK_ARG(run_smem(warps_per_block, games_per_warp) <= (size_t)smem_max,
                 "st_env_set_launch: %d warps x %d games need %zu bytes of shared memory per block (device: %d)",
                 warps_per_block, games_per_warp, run_smem(warps_per_block, games_per_warp), smem_max);
    int occ = 0;
    ST_CUDA(run_occupancy(warps_per_block, games_per_warp, &occ));
    ST_CHECK_ARG(occ >= 1, "st_env_set_launch: %d warps per block do not fit on an SM", warps_per_block);
    e->wpb = warps_per_block;
    e->gpw = games_per_warp;
    e->max_bps = occ;
    e->bps = blocks_per_sm == 0 ? occ : std::min(blocks_per_sm, occ);
    e->gpf = games_per_fetch;
    if (e->graph) { cudaGraphExecDestroy(e->graph); e->graph = nullptr; }
    return ST_OK;
}

extern "C" st_status st_env_get_launch(st_env* e, int32_t* out)
{
    ST_CHECK_ARG(e && out, "st_env_get_launch: null argument");
    out[0] = e->wpb;
    out[1] = e->bps > 0 ? e->bps : std::max(1, e->max_bps);
    out[2] = e->gpw;
    out[3] = e->gpf;
    return ST_OK;
}

extern "C" st_status st_env_run(st_env* e, int32_t n_steps, int32_t ring_steps, int16_t* action_ring,
                                int8_t* reward_ring, uint8_t* done_ring, int16_t* ply_ring, uint8_t* mask_ring)
{
    ST_NVTX("st_env_run");
    ST_CHECK_ARG(e, "st_env_run: null env");
    ST_CHECK_ARG(n_steps >= 0, "st_env_run: n_steps < 0");
    ST_CHECK_ARG(ring_steps >= 1, "st_env_run: ring_steps must be >= 1");
    ST_CHECK_ARG(!mask_ring || aligned16(mask_ring), "st_env_run: mask_ring must be 16-byte aligned");
    if (n_steps == 0) return ST_OK;
    DeviceGuard guard(e->device);
    const int bps = e->bps > 0 ? e->bps : std::max(1, e->max_bps);
    const int64_t key[11] = {n_steps, ring_steps, (int64_t)action_ring, (int64_t)reward_ring, (int64_t)done_ring,
                             (int64_t)ply_ring, (int64_t)mask_ring, e->wpb, bps, e->gpf, e->gpw};
    const int per_block = e->wpb * e->gpw;
    const int blocks = std::max(1, std::min(e->sms * bps, (e->N + per_block - 1) / per_block));
    const int nsplit = parts_per_slot(e->N, blocks * per_block, n_steps);
    EnvArgs a = env_args(e);
    // A non-default stream gets the launch pair (queue reset + persistent
    // kernel) captured once into a CUDA graph and replayed afterwards.
    if (e->stream != nullptr) {
        if (e->graph && std::memcmp(key, e->graph_key, sizeof(key)) == 0) {
            ST_CUDA(cudaGraphLaunch(e->graph, e->stream));
            e->now += n_steps;
            return ST_OK;
        }
        if (e->graph) { cudaGraphExecDestroy(e->graph); e->graph = nullptr; }
        cudaGraph_t graph = nullptr;
        ST_CUDA(cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal));
        cudaMemsetAsync(e->queue, 0, sizeof(int32_t), e->stream);
        if (nsplit > 1) cudaMemsetAsync(e->part_done, 0, (size_t)e->N * sizeof(int32_t), e->stream);
        launch_run(e, a, blocks, n_steps, ring_steps, action_ring, reward_ring, done_ring, ply_ring, mask_ring, nsplit);
        if (e->hist) k_env_advance<<<1, 1, 0, e->stream>>>(e->d_now, n_steps);
        const cudaError_t launch_err = cudaGetLastError();
        const cudaError_t cap_err = cudaStreamEndCapture(e->stream, &graph);
        if (launch_err != cudaSuccess || cap_err != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            stg::set_error("st_env_run: capture failed: %s",
                           cudaGetErrorString(launch_err != cudaSuccess ? launch_err : cap_err));
            return ST_ERR_CUDA;
        }
        const cudaError_t inst_err = cudaGraphInstantiate(&e->graph, graph, 0);
        cudaGraphDestroy(graph);
        if (inst_err != cudaSuccess) {
            e->graph = nullptr;
            stg::set_error("st_env_run: graph instantiate failed: %s", cudaGetErrorString(inst_err));
            return ST_ERR_CUDA;
        }
        std::memcpy(e->graph_key, key, sizeof(key));
        ST_CUDA(cudaGraphLaunch(e->graph, e->stream));
        e->now += n_steps;
        return ST_OK;
    }
    ST_CUDA(cudaMemsetAsync(e->queue, 0, sizeof(int32_t), e->stream));
    if (nsplit > 1) ST_CUDA(cudaMemsetAsync(e->part_done, 0, (size_t)e->N * sizeof(int32_t), e->stream));
    launch_run(e, a, blocks, n_steps, ring_steps, action_ring, reward_ring, done_ring, ply_ring, mask_ring, nsplit);
    ST_CUDA(cudaGetLastError());
    if (e->hist) {
        k_env_advance<<<1, 1, 0, e->stream>>>(e->d_now, n_steps);
        ST_CUDA(cudaGetLastError());
    }
    e->now += n_steps;
    return ST_OK;
}

extern "C" st_status st_env_sync(st_env* e)
{
    ST_NVTX("st_env_sync");
    ST_CHECK_ARG(e, "st_env_sync: null env");
    DeviceGuard guard(e->device);
    int32_t h[2];
    ST_CUDA(cudaMemcpyAsync(h, e->status, sizeof(h), cudaMemcpyDeviceToHost, e->stream));
    ST_CUDA(cudaStreamSynchronize(e->stream));
    if (h[0] != 0) {
        const int32_t init_status[2] = {0, 0x7FFFFFFF};
        ST_CUDA(cudaMemcpyAsync(e->status, init_status, sizeof(init_status), cudaMemcpyHostToDevice, e->stream));
        ST_CUDA(cudaStreamSynchronize(e->stream));
        stg::set_error("device error latched: code %d, first index %d", h[0], h[1]);
        return (st_status)h[0];
    }
    return ST_OK;
}

extern "C" st_status st_env_stats(st_env* e, uint32_t* stats_out)
{
    ST_NVTX("st_env_stats");
    ST_CHECK_ARG(e && stats_out, "st_env_stats: null argument");
    DeviceGuard guard(e->device);
    ST_CUDA(cudaMemcpyAsync(stats_out, e->stats, (size_t)e->N * 8 * sizeof(uint32_t), cudaMemcpyDeviceToDevice,
                            e->stream));
    return ST_OK;
}

extern "C" st_status st_env_export(st_env* e, const int32_t* idx, int32_t n, st_position* out)
{
    ST_NVTX("st_env_export");
    ST_CHECK_ARG(e && (n == 0 || (idx && out)), "st_env_export: null argument");
    ST_CHECK_ARG(n >= 0, "st_env_export: n < 0");
    if (n == 0) return ST_OK;
    DeviceGuard guard(e->device);
    EnvArgs a = env_args(e);
    const int blocks = (n + kPlainWarps - 1) / kPlainWarps;
    k_env_export<<<blocks, 32 * kPlainWarps, kPlainWarps * sizeof(SmemGame), e->stream>>>(a, idx, n, out);
    ST_CUDA(cudaGetLastError());
    return ST_OK;
}

extern "C" st_status st_env_import(st_env* e, const int32_t* idx, int32_t n, const st_position* in)
{
    ST_NVTX("st_env_import");
    ST_CHECK_ARG(e && (n == 0 || (idx && in)), "st_env_import: null argument");
    ST_CHECK_ARG(n >= 0, "st_env_import: n < 0");
    if (n == 0) return ST_OK;
    DeviceGuard guard(e->device);
    EnvArgs a = env_args(e);
    const int blocks = (n + kPlainWarps - 1) / kPlainWarps;
    k_env_import<<<blocks, 32 * kPlainWarps, kPlainWarps * sizeof(SmemGame), e->stream>>>(a, idx, n, in);
    ST_CUDA(cudaGetLastError());
    return ST_OK;
}

extern "C" st_status st_env_set_setup_pool(st_env* e, const uint8_t* pool, int32_t M, uint32_t flags)
{
    ST_NVTX("st_env_set_setup_pool");
    ST_CHECK_ARG(e, "st_env_set_setup_pool: null env");
    ST_CHECK_ARG(M >= 0 && M <= ST_MAX_POOL, "st_env_set_setup_pool: M must be in [0, %d]", ST_MAX_POOL);
    ST_CHECK_ARG((flags & ~ST_POOL_MIRROR) == 0, "st_env_set_setup_pool: unknown flags");
    ST_CHECK_ARG(M == 0 || pool, "st_env_set_setup_pool: null pool");
    DeviceGuard guard(e->device);
    uint8_t* dev = nullptr;
    if (M > 0) {
        const size_t bytes = (size_t)2 * (size_t)M * 40;
        std::vector<uint8_t> h(bytes);
        ST_CUDA(cudaMemcpyAsync(h.data(), pool, bytes, cudaMemcpyDeviceToHost, e->stream));
        ST_CUDA(cudaStreamSynchronize(e->stream));
        static const int want[12] = {1, 8, 5, 4, 4, 4, 3, 2, 1, 1, 1, 6};
        for (size_t k = 0; k < (size_t)2 * (size_t)M; ++k) {
            int cnt[12] = {0};
            bool ok = true;
            for (int i = 0; i < 40 && ok; ++i) {
                const uint8_t t = h[k * 40 + i];
                if (t >= 12) ok = false;
                else cnt[t]++;
            }
            for (int t = 0; t < 12 && ok; ++t) ok = cnt[t] == want[t];
            ST_CHECK_ARG(ok, "st_env_set_setup_pool: side %d entry %d is not one side's 40 pieces", (int)(k / M),
                         (int)(k % M));
        }
        cudaError_t err = cudaMalloc(&dev, bytes);
        if (err == cudaSuccess) err = cudaMemcpyAsync(dev, h.data(), bytes, cudaMemcpyHostToDevice, e->stream);
        if (err == cudaSuccess) err = cudaStreamSynchronize(e->stream);
        if (err != cudaSuccess) {
            cudaFree(dev);
            stg::set_error("st_env_set_setup_pool: %s", cudaGetErrorString(err));
            return err == cudaErrorMemoryAllocation ? ST_ERR_OOM : ST_ERR_CUDA;
        }
    }
    ST_CUDA(cudaStreamSynchronize(e->stream));   // no launch still reads the old pool
    cudaFree(e->pool);
    e->pool = dev;
    e->pool_m = M;
    e->pool_flags = flags;
    e->cfg_floor = e->now;
    if (e->graph) { cudaGraphExecDestroy(e->graph); e->graph = nullptr; }
    return ST_OK;
}

extern "C" st_status st_env_pin(st_env* e, const int32_t* idx, int32_t n, const st_position* states)
{
    ST_NVTX("st_env_pin");
    ST_CHECK_ARG(e, "st_env_pin: null env");
    ST_CHECK_ARG(n >= 0 && n <= e->N, "st_env_pin: n must be in [0, N]");
    ST_CHECK_ARG(n == 0 || (idx && states), "st_env_pin: null argument");
    DeviceGuard guard(e->device);
    ST_CUDA(cudaStreamSynchronize(e->stream));   // no launch still reads the old pin set
    if (!e->pin_of) {
        cudaError_t err = cudaMalloc(&e->pin_of, (size_t)e->N * sizeof(int32_t));
        if (err != cudaSuccess) {
            e->pin_of = nullptr;
            stg::set_error("st_env_pin: %s", cudaGetErrorString(err));
            return ST_ERR_OOM;
        }
    }
    cudaFree(e->pins);
    e->pins = nullptr;
    e->n_pins = 0;
    e->cfg_floor = e->now;
    if (e->graph) { cudaGraphExecDestroy(e->graph); e->graph = nullptr; }
    ST_CUDA(cudaMemsetAsync(e->pin_of, 0xFF, (size_t)e->N * sizeof(int32_t), e->stream));
    if (n == 0) return ST_OK;
    RootState* recs = nullptr;
    cudaError_t err = cudaMalloc(&recs, (size_t)n * sizeof(RootState));
    if (err != cudaSuccess) {
        stg::set_error("st_env_pin: %s", cudaGetErrorString(err));
        return ST_ERR_OOM;
    }
    EnvArgs a = env_args(e);
    const int blocks = (n + kPlainWarps - 1) / kPlainWarps;
    k_env_pin<<<blocks, 32 * kPlainWarps, kPlainWarps * sizeof(RolloutSmem), e->stream>>>(a, idx, n, states, recs,
                                                                                          e->pin_of);
    err = cudaGetLastError();
    if (err != cudaSuccess) {
        cudaStreamSynchronize(e->stream);
        cudaFree(recs);
        stg::set_error("st_env_pin: launch failed: %s", cudaGetErrorString(err));
        return ST_ERR_CUDA;
    }
    e->pins = recs;
    e->n_pins = n;
    return ST_OK;
}

extern "C" st_status st_env_enable_history(st_env* e, int32_t H)
{
    ST_NVTX("st_env_enable_history");
    ST_CHECK_ARG(e, "st_env_enable_history: null env");
    ST_CHECK_ARG(H >= 0 && H <= ST_MAX_HISTORY, "st_env_enable_history: H must be in [0, %d]", ST_MAX_HISTORY);
    DeviceGuard guard(e->device);
    ST_CUDA(cudaStreamSynchronize(e->stream));   // no launch still writes the old ring
    if (e->graph) { cudaGraphExecDestroy(e->graph); e->graph = nullptr; }
    cudaFree(e->hist);
    e->hist = nullptr;
    e->H = 0;
    if (H == 0) return ST_OK;
    cudaError_t err = cudaSuccess;
    if (!e->d_now) err = cudaMalloc(&e->d_now, sizeof(long long));
    if (err == cudaSuccess) err = cudaMalloc(&e->hist, (size_t)H * (size_t)e->N * sizeof(uint32_t));
    if (err != cudaSuccess) {
        e->hist = nullptr;
        cudaGetLastError();
        stg::set_error("st_env_enable_history: %zu bytes: %s", (size_t)H * (size_t)e->N * sizeof(uint32_t),
                       cudaGetErrorString(err));
        return ST_ERR_OOM;
    }
    const long long now = e->now;
    ST_CUDA(cudaMemcpyAsync(e->d_now, &now, sizeof(now), cudaMemcpyHostToDevice, e->stream));
    // start marks left from before are stale once steps were taken unrecorded
    if (now > 0) k_env_clear_marks<<<(e->N + 255) / 256, 256, 0, e->stream>>>(e->core, e->N);
    ST_CUDA(cudaGetLastError());
    ST_CUDA(cudaStreamSynchronize(e->stream));
    e->H = H;
    e->hist_start = now;
    return ST_OK;
}

extern "C" st_status st_env_current_step(st_env* e, int64_t* now)
{
    ST_NVTX("st_env_current_step");
    ST_CHECK_ARG(e && now, "st_env_current_step: null argument");
    *now = e->now;
    return ST_OK;
}

static st_status hist_window(st_env* e, int64_t t, bool need_row, const char* fn)
{
    ST_CHECK_ARG(e, "%s: null env", fn);
    ST_CHECK_ARG(e->hist, "%s: the history is off (st_env_enable_history)", fn);
    const long long lo = std::max(e->hist_start, e->now - (long long)e->H);
    const long long hi = need_row ? e->now - 1 : e->now;
    ST_CHECK_ARG(t >= lo && t <= hi, "%s: step %lld outside the window [%lld, %lld]", fn, (long long)t, lo, hi);
    return ST_OK;
}

extern "C" st_status st_env_history_positions(st_env* e, int64_t t, st_position* out, uint8_t* status,
                                              uint8_t* ended, int32_t* since)
{
    ST_NVTX("st_env_history_positions");
    const st_status w = hist_window(e, t, false, "st_env_history_positions");
    if (w != ST_OK) return w;
    ST_CHECK_ARG(out, "st_env_history_positions: null out");
    DeviceGuard guard(e->device);
    EnvArgs a = env_args(e);
    // teams of kHistLanes lanes (32 / kHistLanes slots per warp), their chase
    // stores in a stream-ordered scratch array
    constexpr int kHistLanes = 4, kHistWarps = 4, kTeams = kHistWarps * 32 / kHistLanes;
    uint64_t* pi = nullptr;
    ST_CUDA(cudaMallocAsync(&pi, (size_t)e->N * kPiWords * sizeof(uint64_t), e->stream));
    const int blocks = (e->N + kTeams - 1) / kTeams;
    k_env_hist_positions<kHistLanes><<<blocks, 32 * kHistWarps, kTeams * sizeof(HistSmem), e->stream>>>(
        a, hist_query(e, t), out, status, ended, since, pi);
    const cudaError_t err = cudaGetLastError();
    cudaFreeAsync(pi, e->stream);
    ST_CUDA(err);
    return ST_OK;
}

extern "C" st_status st_env_history_steps(st_env* e, int64_t t, int16_t* action, uint8_t* done, int8_t* reward,
                                          uint8_t* start)
{
    ST_NVTX("st_env_history_steps");
    const st_status w = hist_window(e, t, true, "st_env_history_steps");
    if (w != ST_OK) return w;
    DeviceGuard guard(e->device);
    k_env_hist_steps<<<(e->N + 255) / 256, 256, 0, e->stream>>>(e->N, hist_query(e, t), action, done, reward, start);
    ST_CUDA(cudaGetLastError());
    return ST_OK;
}

extern "C" st_status st_env_history_logs(st_env* e, int64_t t, int32_t L, uint8_t* setups, int16_t* logs,
                                         int16_t* plies, uint8_t* status)
{
    ST_NVTX("st_env_history_logs");
    const st_status w = hist_window(e, t, false, "st_env_history_logs");
    if (w != ST_OK) return w;
    ST_CHECK_ARG(L >= 1 && L <= 32767, "st_env_history_logs: L must be in [1, 32767]");
    ST_CHECK_ARG(setups && logs && plies, "st_env_history_logs: null argument");
    DeviceGuard guard(e->device);
    EnvArgs a = env_args(e);
    const int blocks = (e->N + kPlainWarps - 1) / kPlainWarps;
    k_env_hist_logs<<<blocks, 32 * kPlainWarps, kPlainWarps * sizeof(SmemGame), e->stream>>>(
        a, hist_query(e, t), L, setups, logs, plies, status);
    ST_CUDA(cudaGetLastError());
    return ST_OK;
}

extern "C" st_status st_env_sample_actions(st_env* e, int16_t* actions)
{
    ST_NVTX("st_env_sample_actions");
    ST_CHECK_ARG(e && actions, "st_env_sample_actions: null argument");
    DeviceGuard guard(e->device);
    EnvArgs a = env_args(e);
    const int blocks = (e->N + kPlainWarps - 1) / kPlainWarps;
    k_env_sample<<<blocks, 32 * kPlainWarps, kPlainWarps * sizeof(SmemGame), e->stream>>>(a, actions);
    ST_CUDA(cudaGetLastError());
    return ST_OK;
}
