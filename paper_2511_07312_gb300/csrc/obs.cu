// obs.cu -- replay of action logs into positions and the information-state
// planes of App. C (st_replay_positions, st_obs_encode).
//
// Two kernels.  k_replay: a block of four warps per run of consecutive
// items replays each item's log in shared memory (with full legality checks
// and the history features), continuing from the previous item of the run
// when it is the same game at a later ply, so items sorted by (game, ply)
// walk each log once per run (App. B.1: compact records, states
// reconstructed on demand).  Within a ply the warps split the work on the
// position before the move (the move worked out, its legality, two sets of
// features), so the ply's serial path is the longest of them rather than
// their sum.  It writes the replayed state of every item to a scratch record
// (or an st_position), plus the legal mask.  k_obs_emit: one warp per item
// turns the record into the 487 planes: lane l owns four squares, all lanes
// walk the channels together, and each channel row is one coalesced
// 100-byte uint8 store and one 200-byte bf16 store per warp.
#include <mutex>
#include <atomic>
#include "engine.cuh"
#include "features.cuh"
#include "host_common.h"

using namespace stg;

namespace {

constexpr int kReplayWarps = 4;                    // a replay block: move, legality, two feature warps
constexpr int kEmitWarps = 4;
constexpr int kPlaneBytes = ST_NCHAN * 100;        // 48,700
constexpr int kGroups = ST_NCHAN * 25;             // 4 squares per group

// Replayed state of one item, as the emission kernel needs it.
struct __align__(16) ItemState {
    GameCore c;
    uint16_t hist[32];
    uint64_t fa[kPieces];
    uint64_t fb[kPieces];
};
static_assert(sizeof(ItemState) == 288 + 64 + 1280, "ItemState layout");

struct __align__(16) ReplaySmem {
    SmemGame g;
    FeatSmem f;
    uint64_t pi[kPiWords];
    uint16_t ring[kRing];
    int live, legal;   // the game goes on (warp 0), the action is legal (warp 1): written before the block's barrier
};

struct ReplayArgs {
    const uint8_t* setups;
    const int16_t* actions;
    int log_len;
    int num_logs;
    const int32_t* game;
    const int16_t* ply;
    int B;
    Rules R;
    int items_per_block;
    ItemState* state_out;    // obs mode
    st_position* pos_out;    // position mode
    uint8_t* mask_out;
    uint8_t* status;
};

__device__ __noinline__ bool setup_ok(const uint8_t* s)
{
    int cnt[24];
    for (int i = 0; i < 24; ++i) cnt[i] = 0;
    for (int p = 0; p < 80; ++p) {
        if (s[p] >= 12) return false;
        cnt[(p / 40) * 12 + s[p]]++;
    }
    const int want[12] = {1, 8, 5, 4, 4, 4, 3, 2, 1, 1, 1, 6};
    for (int i = 0; i < 24; ++i)
        if (cnt[i] != want[i % 12]) return false;
    return true;
}

__device__ void write_position(const SmemGame* G, const uint16_t* ring, st_position* o)
{
    const int lane = lane_id();
    uint8_t* ob = reinterpret_cast<uint8_t*>(o);
    for (int b = lane; b < 240; b += 32) ob[b] = reinterpret_cast<const uint8_t*>(&G->c)[b];
    for (int h = lane; h < 256; h += 32) o->hist[h] = (uint16_t)hist_at(G, ring, h);
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
}

// Zeroes n bytes with every thread of the block.
__device__ void zero_block(void* dst, int n)
{
    uint8_t* d = static_cast<uint8_t*>(dst);
    for (int k = threadIdx.x; k < n; k += blockDim.x) d[k] = 0;
}

// Item i's outputs, with every thread of the replay block: its status and,
// as asked, its snapshot or replay record (warp 0) and its legal mask (warp
// 1), or zeros for an invalid item.  Out of line, so that the ply loop's
// registers are allocated alone.
__device__ __noinline__ void item_outputs(const ReplayArgs& A, ReplaySmem* S, int i, bool ok)
{
    SmemGame* G = &S->g;
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    if (threadIdx.x == 0 && A.status) A.status[i] = ok ? 0 : 1;
    if (!ok) {
        if (A.pos_out) zero_block(A.pos_out + i, sizeof(st_position));
        if (A.state_out) zero_block(A.state_out + i, sizeof(ItemState));
        if (A.mask_out) zero_block(A.mask_out + (size_t)i * kMaskBytes, kMaskBytes);
        return;
    }
    if (warp == 0) {
        if (A.pos_out) write_position(G, S->ring, A.pos_out + i);
        if (A.state_out) {
            ItemState* o = A.state_out + i;
            if (lane < 18) reinterpret_cast<uint4*>(&o->c)[lane] = reinterpret_cast<const uint4*>(&G->c)[lane];
            o->hist[lane] = (uint16_t)hist_at(G, S->ring, lane);
            for (int k = lane; k < kPieces; k += 32) { o->fa[k] = S->f.a[k]; o->fb[k] = S->f.b[k]; }
        }
    } else if (warp == 1 && A.mask_out) {
        gen_moves(G, Team<32>(), G->c.ply & 1, A.R.flags, false, true, S->pi,
                  reinterpret_cast<uint32_t*>(A.mask_out + (size_t)i * kMaskBytes));
    }
}

// One block of four warps per run of items_per_block consecutive items
// replays each item's log in shared memory, continuing from the previous
// item of the run when it is the same game at a later ply.  Per ply the
// warps read the position before the move side by side: warp 0 checks that
// the game has not ended and works out the move without writing
// (plan_apply), warp 1 checks the move's legality and records its threats,
// warps 2 and 3 record its other history features (active adjacency;
// evasion and protection); after a block barrier warp 0 writes the move
// (commit_apply).
// At an item the block writes its status and, as asked, its snapshot or
// replay record (warp 0) and its legal mask (warp 1).
__global__ void __launch_bounds__(32 * kReplayWarps) k_replay(ReplayArgs A)
{
    extern __shared__ __align__(16) unsigned char smem[];
    ReplaySmem* S = reinterpret_cast<ReplaySmem*>(smem);
    SmemGame* G = &S->g;
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    const int i0 = blockIdx.x * A.items_per_block;
    const int i1 = min(A.B, i0 + A.items_per_block);
    const bool track = A.state_out != nullptr;
    int cur_game = -1, cur_ply = 0;
    bool valid = false;
    for (int i = i0; i < i1; ++i) {
        const int gi = A.game[i];
        const int p = A.ply[i];
        bool ok = gi >= 0 && gi < A.num_logs && p >= 0 && p <= A.log_len;
        if (ok && !(valid && gi == cur_game && p >= cur_ply)) {
            const uint8_t* setup = A.setups + 80 * (size_t)gi;
            ok = setup_ok(setup);
            if (ok) {
                if (warp == 0) reset_game(G, Team<32>(), 0, 0, 0, 0, setup);
                for (int k = threadIdx.x; k < kPieces; k += blockDim.x) { S->f.a[k] = 0; S->f.b[k] = 0; }
                cur_game = gi;
                cur_ply = 0;
                valid = true;
            } else {
                valid = false;
            }
            __syncthreads();
        }
        if (ok) {
            const int16_t* log = A.actions + (size_t)A.log_len * (size_t)gi;
            while (cur_ply < p) {
                const int a = log[cur_ply];
                const bool in_range = a >= 0 && a < 10000;
                ApplyPlan plan;
                if (warp == 0) {
                    if (lane == 0) {
                        // an intermediate position must not have ended the game
                        S->live = !(cur_ply > 0 && (flag_dead(G, G->c.ply & 1) || G->c.battleless >= A.R.k ||
                                                    G->c.ply >= A.R.cap));
                        if (in_range) plan = plan_apply(G, a);
                    }
                } else if (warp == 1) {
                    const bool legal = move_legal(G, a, A.R.flags, S->ring, S->pi);
                    if (lane == 0) S->legal = legal;
                    // (an illegal action's features are discarded with the item)
                    if (track && in_range && G->board[a / 100] < kPieces)
                        threats_of_move(G, &S->f, a, G->board[a - 100 * (a / 100)] != kEmpty);
                } else if (track && in_range && G->board[a / 100] < kPieces) {
                    if (warp == 2) active_adjacency(G, &S->f, a, A.R.flags);
                    else evasion_protection(G, &S->f, a);
                }
                __syncthreads();
                const bool legal = S->live && S->legal;
                if (warp == 0 && lane == 0 && legal) commit_apply(G, plan, S->ring, S->pi);
                __syncthreads();
                if (!legal) { ok = false; break; }
                ++cur_ply;
            }
            if (!ok) valid = false;
        }
        item_outputs(A, S, i, ok);
        __syncthreads();   // outputs done before the next item's replay changes the game
    }
}

// ---------------------------------------------------------------- emission

struct __align__(16) EmitSmem {
    ItemState s;
    uint8_t board[112];
    uint64_t death[2][100];          // bit 10*(cause-1)+rank per side and square
    uint32_t ratio[2][2][12];        // side x {unmoved, moved} x type: u8 | bf16<<8
    uint32_t frac41, frac42;
};

struct EmitArgs {
    const ItemState* items;
    const uint8_t* status;
    const int8_t* player;
    int B;
    Rules R;
    uint8_t* planes;
    uint16_t* planes_bf16;
};

constexpr uint32_t kOne = 1u | (0x3F80u << 8);
constexpr uint32_t kMinus = 255u | (0xBF80u << 8);
constexpr uint32_t kRatioOne = 255u | (0x3F80u << 8);

// u8 floor(255*num/den + 1/2) | bf16 bits of num/den << 8 (IEEE fp32 division
// then round-to-nearest-even; exact for den <= 1600).
__device__ __forceinline__ uint32_t ratio_code(uint32_t num, uint32_t den)
{
    if (num == 0) return 0u;
    const uint32_t u8 = (510u * num + den) / (2u * den);
    const float q = __fdiv_rn((float)num, (float)den);
    uint32_t bits = __float_as_uint(q);
    bits += 0x7FFFu + ((bits >> 16) & 1u);
    return u8 | ((bits >> 16) << 8);
}

// Channel-major emission: lane l < 25 owns squares 4l .. 4l+3 and keeps what
// its squares need in registers; all lanes walk the 487 channels together
// (no divergence between lanes), each channel row written with one 4-byte
// uint8 store and one 8-byte bf16 store per lane, 100 / 200 contiguous bytes
// per warp.  A cell code is u8 | bf16 << 8.
struct RowOut {
    uint8_t* u8;
    uint16_t* bf;
    int l;       // owning lane (squares 4l .. 4l+3)
    bool on;     // l < 25
    __device__ __forceinline__ void codes(int ch, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3) const
    {
        if (!on) return;
        if (u8)
            *reinterpret_cast<uint32_t*>(u8 + 100 * ch + 4 * l) =
                (c0 & 0xFFu) | ((c1 & 0xFFu) << 8) | ((c2 & 0xFFu) << 16) | ((c3 & 0xFFu) << 24);
        if (bf)
            *reinterpret_cast<uint2*>(bf + 100 * ch + 4 * l) =
                make_uint2((c0 >> 8) | ((c1 >> 8) << 16), (c2 >> 8) | ((c3 >> 8) << 16));
    }
    // cells of value 0 or 1 (u8 1, bf16 1.0)
    __device__ __forceinline__ void bits(int ch, uint32_t b0, uint32_t b1, uint32_t b2, uint32_t b3) const
    {
        packed(ch, b0 | (b1 << 8) | (b2 << 16) | (b3 << 24));
    }
    // the same, the four cells given as the bytes of m (each 0 or 1)
    __device__ __forceinline__ void packed(int ch, uint32_t m) const
    {
        if (!on) return;
        if (u8) *reinterpret_cast<uint32_t*>(u8 + 100 * ch + 4 * l) = m;
        if (bf)
            *reinterpret_cast<uint2*>(bf + 100 * ch + 4 * l) =
                make_uint2(((m & 1u) | ((m << 8) & 0x10000u)) * 0x3F80u,
                           (((m >> 16) & 1u) | ((m >> 8) & 0x10000u)) * 0x3F80u);
    }
    // channels ch0 .. ch0+N-1: bit k of the four squares' words w, eight
    // channels from one gather of the words' k/8-th bytes (byte i of X is
    // square i's)
    // (loops kept rolled: the emission's code would otherwise outgrow the
    // instruction cache)
    template <int N>
    __device__ __forceinline__ void bit_channels(int ch0, const uint64_t (&w)[4]) const
    {
#pragma unroll 1
        for (int k0 = 0; k0 < N; k0 += 8) {
            const uint32_t X = (uint32_t)((w[0] >> k0) & 0xFFu) | ((uint32_t)((w[1] >> k0) & 0xFFu) << 8) |
                               ((uint32_t)((w[2] >> k0) & 0xFFu) << 16) | ((uint32_t)((w[3] >> k0) & 0xFFu) << 24);
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (k0 + k < N) packed(ch0 + k0 + k, (X >> k) & 0x01010101u);
        }
    }
    // rows ch0 .. ch0+N-1 cleared over the lane's four squares
    template <int N>
    __device__ __forceinline__ void zero_rows(int ch0) const
    {
#pragma unroll 4
        for (int k = 0; k < N; ++k) packed(ch0 + k, 0u);
    }
    // cell (row ch, square 4l+i) set to 1; its row was cleared by this lane
    // before (the same thread's later store to the same bytes wins)
    __device__ __forceinline__ void one(int ch, int i) const
    {
        if (!on) return;
        if (u8) u8[100 * ch + 4 * l + i] = 1;
        if (bf) bf[100 * ch + 4 * l + i] = 0x3F80u;
    }
};


__device__ __forceinline__ void emit_planes(const EmitSmem* E, int me, const RowOut& o)
{
    const ItemState& st = E->s;
    const int s0 = o.on ? 4 * o.l : 0;
    int occ[4], side[4], ty[4];
    uint32_t fl[4];
    bool pc[4], mn[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        occ[i] = E->board[s0 + i];
        pc[i] = occ[i] < kPieces;
        side[i] = pc[i] ? occ[i] / 40 : -1;
        mn[i] = side[i] == me;
        fl[i] = pc[i] ? st.c.flags[occ[i]] : 0u;
        ty[i] = pc[i] ? st.c.type[occ[i]] : 0xFF;
    }
    // 0-11: own pieces by type (one channel per square at most)
    o.zero_rows<12>(0);
#pragma unroll
    for (int i = 0; i < 4; ++i)
        if (pc[i] && mn[i] && ty[i] < 12) o.one(ty[i], i);
    // 12-23 (opponent's pieces), 24-35 (own pieces): probability of each type
    for (int g = 0; g < 2; ++g) {
        const int want = g == 0 ? 1 - me : me;
        int kind[4], row[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            kind[i] = (!pc[i] || side[i] != want) ? 0 : ((fl[i] & 2) ? 1 : ((fl[i] & 8) ? 2 : 3));
            row[i] = 2 * (side[i] < 0 ? 0 : side[i]) + ((fl[i] & 4) ? 1 : 0);
        }
        const uint32_t* ratio = &E->ratio[0][0][0];
        for (int T = 0; T < 12; ++T) {
            uint32_t c[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
                c[i] = kind[i] == 1 ? (ty[i] == T ? kRatioOne : 0u)
                     : kind[i] == 2 ? (T == kScout ? kRatioOne : 0u)
                     : kind[i] == 3 ? ratio[12 * row[i] + T] : 0u;
            o.codes(12 + 12 * g + T, c[0], c[1], c[2], c[3]);
        }
    }
    // 36-42
    o.bits(36, pc[0] && mn[0] && !(fl[0] & 2), pc[1] && mn[1] && !(fl[1] & 2), pc[2] && mn[2] && !(fl[2] & 2),
           pc[3] && mn[3] && !(fl[3] & 2));
    o.bits(37, pc[0] && !mn[0] && !(fl[0] & 2), pc[1] && !mn[1] && !(fl[1] & 2), pc[2] && !mn[2] && !(fl[2] & 2),
           pc[3] && !mn[3] && !(fl[3] & 2));
    o.bits(38, occ[0] == kEmpty, occ[1] == kEmpty, occ[2] == kEmpty, occ[3] == kEmpty);
    o.bits(39, pc[0] && mn[0] && (fl[0] & 4), pc[1] && mn[1] && (fl[1] & 4), pc[2] && mn[2] && (fl[2] & 4),
           pc[3] && mn[3] && (fl[3] & 4));
    o.bits(40, pc[0] && !mn[0] && (fl[0] & 4), pc[1] && !mn[1] && (fl[1] & 4), pc[2] && !mn[2] && (fl[2] & 4),
           pc[3] && !mn[3] && (fl[3] & 4));
    o.codes(41, E->frac41, E->frac41, E->frac41, E->frac41);
    o.codes(42, E->frac42, E->frac42, E->frac42, E->frac42);
    // 43-75 / 76-108: history features of the piece on the square (own / opponent)
    for (int g = 0; g < 2; ++g) {
        uint64_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) w[i] = (pc[i] && mn[i] == (g == 0)) ? st.fa[occ[i]] : 0ull;
        o.bit_channels<33>(43 + 33 * g, w);
    }
    // 109-119 / 120-130: captured piece whose start square this is, by type
    for (int g = 0; g < 2; ++g) {
        int idx[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int s = s0 + i;
            const int pid = s < 40 ? s : (s >= 60 ? s - 20 : -1);
            idx[i] = -2;
            if (pid >= 0 && ((pid / 40) == me) == (g == 0) && !(st.c.flags[pid] & 1)) {
                const int t = st.c.type[pid];
                idx[i] = t <= kMarshal ? t : (t == kBomb ? 10 : -1);
            }
        }
        o.zero_rows<11>(109 + 11 * g);
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (idx[i] >= 0) o.one(109 + 11 * g + idx[i], i);
    }
    // 131-190 / 191-250: deaths on the square by cause and rank (own / opponent)
    for (int g = 0; g < 2; ++g) {
        const int want_side = g == 0 ? me : 1 - me;
        uint64_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) w[i] = E->death[want_side][s0 + i];
        o.bit_channels<60>(131 + 60 * g, w);
    }
    // 251-302 / 303-354: further history features (own / opponent)
    for (int g = 0; g < 2; ++g) {
        uint64_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) w[i] = (pc[i] && mn[i] == (g == 0)) ? st.fb[occ[i]] : 0ull;
        o.bit_channels<52>(251 + 52 * g, w);
    }
    // 355-454: the piece on the square started on square ch - 355
    {
        int ss[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) ss[i] = pc[i] ? start_square(occ[i]) : -1;
        o.zero_rows<100>(355);
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (ss[i] >= 0) o.one(355 + ss[i], i);
    }
    // 455-486: the last 32 moves, +1 on the to-square and -1 on the from-square
    for (int j = 0; j < 32; ++j) {
        const int h = st.hist[j];
        uint32_t c[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int s = s0 + i;
            c[i] = h == 0xFFFF ? 0u : (s == h % 100 ? kOne : (s == h / 100 ? kMinus : 0u));
        }
        o.codes(455 + j, c[0], c[1], c[2], c[3]);
    }
}

__global__ void k_obs_emit(EmitArgs A)
{
    extern __shared__ __align__(16) unsigned char smem[];
    EmitSmem* E = reinterpret_cast<EmitSmem*>(smem) + (threadIdx.x >> 5);
    const int lane = lane_id();
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= A.B) return;
    uint8_t* u8 = A.planes ? A.planes + (size_t)b * kPlaneBytes : nullptr;
    uint16_t* bf = A.planes_bf16 ? A.planes_bf16 + (size_t)b * kPlaneBytes : nullptr;
    if (A.status && A.status[b]) {
        for (int g = lane; g < kGroups; g += 32) {
            if (u8) reinterpret_cast<uint32_t*>(u8)[g] = 0u;
            if (bf) reinterpret_cast<uint2*>(bf)[g] = make_uint2(0u, 0u);
        }
        return;
    }
    {
        const uint4* src = reinterpret_cast<const uint4*>(A.items + b);
        uint4* dst = reinterpret_cast<uint4*>(&E->s);
        for (int k = lane; k < (int)(sizeof(ItemState) / 16); k += 32) dst[k] = src[k];
    }
    for (int s = lane; s < 100; s += 32) { E->death[0][s] = 0; E->death[1][s] = 0; }
    __syncwarp();
    for (int s = lane; s < 112; s += 32) E->board[s] = (s < 100 && is_lake(s)) ? kLake : kEmpty;
    __syncwarp();
    for (int p = lane; p < kPieces; p += 32) {
        const uint8_t f = E->s.c.flags[p];
        if (f & 1) {
            E->board[E->s.c.sq[p]] = (uint8_t)p;
        } else {
            const int cause = f >> 4, t = E->s.c.type[p];
            if (cause >= 1 && t <= kMarshal)
                atomicOr(reinterpret_cast<unsigned long long*>(&E->death[p / 40][E->s.c.sq[p]]),
                         1ull << (10 * (cause - 1) + t));
        }
    }
    // remaining counts per side (lanes 0 and 1), then the probability table
    if (lane < 2) {
        const int side = lane;
        int c[12] = {1, 8, 5, 4, 4, 4, 3, 2, 1, 1, 1, 6};
        int nS = 0, nM = 0, nU = 0;
        for (int k = 0; k < 40; ++k) {
            const int p = side * 40 + k;
            const uint8_t f = E->s.c.flags[p];
            if (!(f & 1) || (f & 2)) { c[E->s.c.type[p]]--; continue; }
            if (f & 8) nS++;
            else if (f & 4) nM++;
            else nU++;
        }
        c[kScout] -= nS;
        const int bimm = c[kFlag] + c[kBomb];
        int m = 0;
        for (int t = 0; t <= kMarshal; ++t) m += c[t];
        for (int t = 0; t < 12; ++t) {
            uint32_t unm = 0, mov = 0;
            if (t == kFlag || t == kBomb) {
                if (nU > 0) unm = ratio_code((uint32_t)c[t], (uint32_t)nU);
            } else {
                if (m > 0) mov = ratio_code((uint32_t)c[t], (uint32_t)m);
                if (nU > 0 && m > 0) unm = ratio_code((uint32_t)((nU - bimm) * c[t]), (uint32_t)(nU * m));
            }
            E->ratio[side][0][t] = unm;
            E->ratio[side][1][t] = mov;
        }
    }
    if (lane == 2) {
        E->frac41 = ratio_code((uint32_t)E->s.c.ply, (uint32_t)A.R.cap);
        E->frac42 = ratio_code((uint32_t)E->s.c.battleless, (uint32_t)A.R.k);
    }
    __syncwarp();
    const int me = (A.player && A.player[b] >= 0) ? (A.player[b] & 1) : (E->s.c.ply & 1);
    RowOut o;
    o.u8 = u8;
    o.bf = bf;
    o.l = lane;
    o.on = lane < 25;
    emit_planes(E, me, o);
}

ReplayArgs replay_args(const uint8_t* setups, const int16_t* actions, int32_t log_len, int32_t num_logs,
                       const int32_t* game, const int16_t* ply, int32_t B, const st_rules* rules)
{
    ReplayArgs a{};
    a.setups = setups; a.actions = actions; a.log_len = log_len; a.num_logs = num_logs;
    a.game = game; a.ply = ply; a.B = B;
    a.R.k = rules->battleless_limit; a.R.cap = rules->max_plies; a.R.flags = rules->flags;
    a.items_per_block = 32;
    return a;
}

std::atomic<int> g_items_per_block{32};   // fastest measured on GB300 for 16,384 items of 64 logs

}  // namespace

extern "C" st_status st_replay_set_chunk(int32_t items_per_block)
{
    ST_NVTX("st_replay_set_chunk");
    ST_CHECK_ARG(items_per_block >= 1 && items_per_block <= 65536, "st_replay_set_chunk: 1..65536");
    g_items_per_block.store(items_per_block);
    return ST_OK;
}

extern "C" st_status st_replay_positions(const uint8_t* setups, const int16_t* actions, int32_t log_len,
                                         int32_t num_logs, const int32_t* game, const int16_t* ply, int32_t B,
                                         const st_rules* rules, st_position* out, uint8_t* item_status,
                                         void* stream)
{
    ST_NVTX("st_replay_positions");
    ST_CHECK_ARG(rules_ok(rules), "st_replay_positions: invalid rules");
    ST_CHECK_ARG(B >= 0 && log_len >= 0 && num_logs >= 0, "st_replay_positions: negative size");
    if (B == 0) return ST_OK;
    ST_CHECK_ARG(setups && actions && game && ply && out, "st_replay_positions: null argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    ReplayArgs a = replay_args(setups, actions, log_len, num_logs, game, ply, B, rules);
    a.items_per_block = g_items_per_block.load();
    a.pos_out = out;
    a.status = item_status;
    const int blocks = (B + a.items_per_block - 1) / a.items_per_block;
    k_replay<<<blocks, 32 * kReplayWarps, sizeof(ReplaySmem), s>>>(a);
    ST_CUDA(cudaGetLastError());
    return ST_OK;
}

extern "C" st_status st_obs_encode(const uint8_t* setups, const int16_t* actions, int32_t log_len, int32_t num_logs,
                                   const int32_t* game, const int16_t* ply, const int8_t* player, int32_t B,
                                   const st_rules* rules, uint8_t* planes, uint16_t* planes_bf16, uint8_t* mask,
                                   uint8_t* item_status, void* stream)
{
    ST_NVTX("st_obs_encode");
    ST_CHECK_ARG(rules_ok(rules), "st_obs_encode: invalid rules");
    ST_CHECK_ARG(B >= 0 && log_len >= 0 && num_logs >= 0, "st_obs_encode: negative size");
    if (B == 0) return ST_OK;
    ST_CHECK_ARG(setups && actions && game && ply, "st_obs_encode: null argument");
    ST_CHECK_ARG(!planes || ((uintptr_t)planes & 3u) == 0, "st_obs_encode: planes must be 4-byte aligned");
    ST_CHECK_ARG(!planes_bf16 || ((uintptr_t)planes_bf16 & 7u) == 0, "st_obs_encode: planes_bf16 must be 8-byte aligned");
    ST_CHECK_ARG(!mask || aligned16(mask), "st_obs_encode: mask must be 16-byte aligned");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const bool need_planes = planes || planes_bf16;
    ItemState* scratch = nullptr;
    uint8_t* status = item_status;
    uint8_t* own_status = nullptr;
    if (need_planes) {
        ST_CUDA(cudaMallocAsync(&scratch, (size_t)B * sizeof(ItemState), s));
        if (!status) {
            const cudaError_t e2 = cudaMallocAsync(&own_status, (size_t)B, s);
            if (e2 != cudaSuccess) cudaFreeAsync(scratch, s);   // the scratch is not left behind
            ST_CUDA(e2);
            status = own_status;
        }
    }
    ReplayArgs a = replay_args(setups, actions, log_len, num_logs, game, ply, B, rules);
    a.items_per_block = g_items_per_block.load();
    a.state_out = scratch;
    a.mask_out = mask;
    a.status = status;
    if (!need_planes && !mask && !status) return ST_OK;
    const int blocks = (B + a.items_per_block - 1) / a.items_per_block;
    k_replay<<<blocks, 32 * kReplayWarps, sizeof(ReplaySmem), s>>>(a);
    cudaError_t err = cudaGetLastError();
    if (err == cudaSuccess && need_planes) {
        EmitArgs e{};
        e.items = scratch; e.status = status; e.player = player; e.B = B; e.R = a.R;
        e.planes = planes; e.planes_bf16 = planes_bf16;
        const int eblocks = (B + kEmitWarps - 1) / kEmitWarps;
        k_obs_emit<<<eblocks, 32 * kEmitWarps, kEmitWarps * sizeof(EmitSmem), s>>>(e);
        err = cudaGetLastError();
    }
    if (scratch) cudaFreeAsync(scratch, s);
    if (own_status) cudaFreeAsync(own_status, s);
    if (err != cudaSuccess) {
        stg::set_error("st_obs_encode: launch failed: %s", cudaGetErrorString(err));
        return ST_ERR_CUDA;
    }
    return ST_OK;
}

// ---------------------------------------------------------------- allocation-free variant
// Same computation as st_obs_encode, for callers that must not allocate
// device memory once they are running.  The per-item replay records live in
// a fixed array in this library's device image instead of a per-call
// stream-ordered allocation.  The paper has no counterpart of this entry
// point.

static __device__ __align__(256) ItemState g_obs_static_items[ST_OBS_STATIC_MAX_ITEMS];
static __device__ __align__(256) uint8_t g_obs_static_status[ST_OBS_STATIC_MAX_ITEMS];

namespace {

constexpr int kMaxDevices = 64;

struct StaticScratch {
    ItemState* items = nullptr;
    uint8_t* status = nullptr;
    bool ready = false;
};

std::mutex g_static_mu;
StaticScratch g_static[kMaxDevices];

// Device addresses of the static arrays on the current device, looked up
// once per device.  The host-side names of the arrays are stand-ins, never
// device addresses; only the looked-up pointers reach a kernel.
st_status static_scratch(StaticScratch* out)
{
    int dev = -1;
    ST_CUDA(cudaGetDevice(&dev));
    ST_CHECK_ARG(dev >= 0 && dev < kMaxDevices, "st_obs_encode_static: device %d beyond %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_static_mu);
    StaticScratch& s = g_static[dev];
    if (!s.ready) {
        void* items = nullptr;
        void* status = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&items, g_obs_static_items);
        if (e == cudaSuccess) e = cudaGetSymbolAddress(&status, g_obs_static_status);
        if (e != cudaSuccess) {
            stg::set_error("st_obs_encode_static: cudaGetSymbolAddress failed on device %d: %s", dev,
                           cudaGetErrorString(e));
            return ST_ERR_CUDA;
        }
        s.items = static_cast<ItemState*>(items);
        s.status = static_cast<uint8_t*>(status);
        s.ready = true;
    }
    *out = s;
    return ST_OK;
}

}  // namespace

extern "C" st_status st_obs_encode_static(const uint8_t* setups, const int16_t* actions, int32_t log_len,
                                          int32_t num_logs, const int32_t* game, const int16_t* ply,
                                          const int8_t* player, int32_t B, const st_rules* rules, uint8_t* planes,
                                          uint16_t* planes_bf16, uint8_t* mask, uint8_t* item_status, void* stream)
{
    ST_NVTX("st_obs_encode_static");
    ST_CHECK_ARG(rules_ok(rules), "st_obs_encode_static: invalid rules");
    ST_CHECK_ARG(B >= 0 && log_len >= 0 && num_logs >= 0, "st_obs_encode_static: negative size");
    ST_CHECK_ARG(B <= ST_OBS_STATIC_MAX_ITEMS,
                 "st_obs_encode_static: %d items exceed the fixed scratch of %d items; split the batch or use "
                 "st_obs_encode", B, ST_OBS_STATIC_MAX_ITEMS);
    if (B == 0) return ST_OK;
    ST_CHECK_ARG(setups && actions && game && ply, "st_obs_encode_static: null argument");
    ST_CHECK_ARG(!planes || ((uintptr_t)planes & 3u) == 0, "st_obs_encode_static: planes must be 4-byte aligned");
    ST_CHECK_ARG(!planes_bf16 || ((uintptr_t)planes_bf16 & 7u) == 0,
                 "st_obs_encode_static: planes_bf16 must be 8-byte aligned");
    ST_CHECK_ARG(!mask || aligned16(mask), "st_obs_encode_static: mask must be 16-byte aligned");
    StaticScratch sc;
    const st_status ss = static_scratch(&sc);
    if (ss != ST_OK) return ss;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const bool need_planes = planes || planes_bf16;
    uint8_t* status = item_status ? item_status : (need_planes ? sc.status : nullptr);
    if (!need_planes && !mask && !status) return ST_OK;
    // k_replay writes every record and status byte of items 0..B-1 before
    // k_obs_emit reads them, so nothing left by an earlier call is read and
    // nothing needs clearing first.
    ReplayArgs a = replay_args(setups, actions, log_len, num_logs, game, ply, B, rules);
    a.items_per_block = g_items_per_block.load();
    a.state_out = need_planes ? sc.items : nullptr;
    a.mask_out = mask;
    a.status = status;
    const int blocks = (B + a.items_per_block - 1) / a.items_per_block;
    k_replay<<<blocks, 32 * kReplayWarps, sizeof(ReplaySmem), s>>>(a);
    cudaError_t err = cudaGetLastError();
    if (err == cudaSuccess && need_planes) {
        EmitArgs e{};
        e.items = sc.items; e.status = status; e.player = player; e.B = B; e.R = a.R;
        e.planes = planes; e.planes_bf16 = planes_bf16;
        const int eblocks = (B + kEmitWarps - 1) / kEmitWarps;
        k_obs_emit<<<eblocks, 32 * kEmitWarps, kEmitWarps * sizeof(EmitSmem), s>>>(e);
        err = cudaGetLastError();
    }
    if (err != cudaSuccess) {
        stg::set_error("st_obs_encode_static: launch failed: %s", cudaGetErrorString(err));
        return ST_ERR_CUDA;
    }
    return ST_OK;
}
