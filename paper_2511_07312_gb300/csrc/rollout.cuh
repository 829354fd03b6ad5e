// rollout.cuh -- shared device code of the search path (App. E "Search",
// steps 1-2): the hidden-piece plan of a position, one belief sample, the
// root state of a position kept in HBM, and one team's rollout from a sample
// (plain, or with the search's forced first move).  Used by st_rollout and
// st_search (search.cu), by the serving engine (serve.cu) and for pinned
// restarts (env.cu).
#pragma once
#include "engine.cuh"
#include "snapshot.cuh"

namespace stg {

// Hidden-piece structure of one position, from the player to move.
struct __align__(16) BeliefPlan {
    uint8_t known[40];      // type of opponent piece i if public, else 0xFF
    uint8_t order[40];      // hidden pieces in ascending square order
    uint8_t is_unmoved[40]; // per entry of order
    uint8_t movable[40];    // sorted movable multiset still to place
    int n_hidden, n_unmoved, n_flag, n_imm, n_mov;
    int opp;
};

// Single thread.
__device__ inline void make_plan(const SmemGame* G, BeliefPlan* B)
{
    const int opp = 1 - (G->c.ply & 1);
    int c[12] = {1, 8, 5, 4, 4, 4, 3, 2, 1, 1, 1, 6};
    int nS = 0;
    for (int k = 0; k < 40; ++k) {
        const int p = opp * 40 + k;
        const uint8_t f = G->c.flags[p];
        if (!(f & 1) || (f & 2)) { B->known[k] = G->c.type[p]; c[G->c.type[p]]--; }
        else if (f & 8) { B->known[k] = kScout; nS++; }
        else B->known[k] = 0xFF;
    }
    c[kScout] -= nS;
    int nh = 0, nu = 0;
    for (int s = 0; s < 100; ++s) {
        const uint8_t p = G->board[s];
        if (p >= kPieces || (int)(p / 40) != opp) continue;
        const int k = p - 40 * opp;
        if (B->known[k] != 0xFF) continue;
        B->order[nh] = (uint8_t)k;
        B->is_unmoved[nh] = (G->c.flags[p] & 4) ? 0 : 1;
        nu += B->is_unmoved[nh];
        nh++;
    }
    int nm = 0;
    for (int t = 0; t <= kMarshal; ++t)
        for (int j = 0; j < c[t] && nm < 40; ++j) B->movable[nm++] = (uint8_t)t;
    B->n_hidden = nh;
    B->n_unmoved = nu;
    B->n_flag = c[kFlag];
    B->n_imm = c[kFlag] + c[kBomb];
    B->n_mov = nm;
    B->opp = opp;
}

// One sample (single thread): the types of opponent pieces 0..39.  Draw w is
// word w%4 of Philox at counter (stream, sample, 0, 3<<24 | w/4).
__device__ inline void draw_sample(const BeliefPlan* B, uint32_t k0, uint32_t k1, uint32_t stream, uint32_t sample,
                                   uint8_t* out)
{
    uint32_t w = 0;
    uint4 buf = make_uint4(0, 0, 0, 0);
    auto next = [&]() -> uint32_t {
        if ((w & 3) == 0) buf = philox(make_uint4(stream, sample, 0u, (3u << 24) | (w >> 2)), k0, k1);
        const uint32_t r = (w & 3) == 0 ? buf.x : (w & 3) == 1 ? buf.y : (w & 3) == 2 ? buf.z : buf.w;
        ++w;
        return r;
    };
    for (int k = 0; k < 40; ++k) out[k] = B->known[k];
    // 1. immovable pieces onto n_imm of the unmoved hidden pieces (partial Fisher-Yates)
    uint8_t idx[40], imm[40];
    const int nu = B->n_unmoved;
    for (int i = 0; i < nu; ++i) { idx[i] = (uint8_t)i; imm[i] = 0xFF; }
    for (int i = 0; i < B->n_imm && i < nu; ++i) {
        const int j = i + (int)uniform_below(next(), (uint32_t)(nu - i));
        const uint8_t t = idx[i]; idx[i] = idx[j]; idx[j] = t;
        imm[idx[i]] = (uint8_t)(i < B->n_flag ? kFlag : kBomb);
    }
    // 2. the movable multiset over the remaining hidden pieces (full Fisher-Yates)
    uint8_t arr[40];
    const int m = B->n_mov;
    for (int i = 0; i < m; ++i) arr[i] = B->movable[i];
    for (int i = m - 1; i >= 1; --i) {
        const int j = (int)uniform_below(next(), (uint32_t)(i + 1));
        const uint8_t t = arr[i]; arr[i] = arr[j]; arr[j] = t;
    }
    int u = 0, nxt = 0;
    for (int h = 0; h < B->n_hidden; ++h) {
        const int k = B->order[h];
        if (B->is_unmoved[h]) {
            const uint8_t t = imm[u++];
            if (t != 0xFF) { out[k] = t; continue; }
        }
        if (nxt < m) out[k] = arr[nxt];
        ++nxt;
    }
}

// Root of a search: the imported position as the rollout warps need it.
struct __align__(16) RootState {
    GameCore c;
    uint8_t board[112];
    uint64_t pi[kPiWords];
    uint16_t ring[kRing];
    BeliefPlan plan;
    int32_t bad;
    int32_t pad[3];
};

struct __align__(16) RolloutSmem {
    SmemGame g;
    uint64_t pi[kPiWords];
    uint16_t ring[kRing];
    uint8_t types[48];
    uint32_t mask[kMaskWordsAlloc];   // a legal mask when a kernel needs one in shared memory
};

// A rollout team's shared-memory record when no history ring is kept; its
// chase store lives in a global scratch slot of the team (the newest four
// entries are cached in the game record), which halves the shared memory a
// rollout needs and doubles the teams an SM can hold.
struct __align__(16) FlatSmem {
    SmemGame g;
    uint8_t types[48];
};

// Warp: import snapshot `in` and write its root state; returns (to every
// lane) and records bad != 0 if the snapshot is invalid.
__device__ inline int build_root(RolloutSmem* S, const st_position* in, RootState* out)
{
    const int lane = lane_id();
    const int bad = import_position(&S->g, in, S->ring, S->pi);
    if (lane == 0) {
        out->bad = bad;
        if (!bad) make_plan(&S->g, &out->plan);
    }
    if (bad) return bad;
    {
        const uint4* src = reinterpret_cast<const uint4*>(&S->g);   // core + board
        uint4* dst = reinterpret_cast<uint4*>(out);
        for (int i = lane; i < (288 + 112) / 16; i += 32) dst[i] = src[i];
    }
    for (int i = lane; i < kRing; i += 32) out->ring[i] = S->ring[i];
    for (int i = lane; i < 2 * S->g.c.n_pi; i += 32) out->pi[i] = S->pi[i];
    return 0;
}

// Team: the rollout record of one belief sample.  Copies root R into G
// (core, board, chase store; the history ring too when `ring` is given),
// puts sample `k` (types given, or drawn from plan) on the opponent's hidden
// pieces and rebuilds the square sets.  types_s: 40 bytes of shared scratch.
template <int L>
__device__ __forceinline__ void begin_rollout(SmemGame* G, uint8_t* types_s, uint64_t* pi, uint16_t* ring,
                                              const Team<L>& T, const RootState* R, const BeliefPlan* plan,
                                              const uint8_t* types, uint32_t k0, uint32_t k1, uint32_t stream,
                                              uint32_t k)
{
    const int lane = T.tl;
    {
        const uint4* src = reinterpret_cast<const uint4*>(R);
        uint4* dst = reinterpret_cast<uint4*>(G);
        for (int i = lane; i < (288 + 112) / 16; i += L) dst[i] = src[i];
        if (ring) {
            const uint4* rs = reinterpret_cast<const uint4*>(R->ring);
            uint4* rd = reinterpret_cast<uint4*>(ring);
            for (int i = lane; i < kRing * 2 / 16; i += L) rd[i] = rs[i];
        }
    }
    T.sync();
    const int npi = G->c.n_pi;
    for (int i = lane; i < 2 * npi; i += L) pi[i] = R->pi[i];
    const int opp = 1 - (G->c.ply & 1);
    if (types) {
        for (int i = lane; i < 40; i += L) types_s[i] = types[i];
    } else if (lane == 0) {
        draw_sample(plan, k0, k1, stream, k, types_s);
    }
    T.sync();
    for (int i = lane; i < 40; i += L) G->c.type[opp * 40 + i] = types_s[i];
    T.sync();
    derive_state(G, ring ? ring : R->ring, pi, T);   // square sets and flag ids of the sampled types
}

__device__ __forceinline__ int tally_slot(int code, int winner, int searcher)
{
    return !code ? 3 : (winner < 0 ? 2 : (winner == searcher ? 0 : 1));
}

// Team: one rollout of `depth` plies of the rollout policy (uniform, or the
// magnet policy under kMagnet) from root R with sample `k`
// (types given, or drawn from plan, R's plan) in the game record G; types_s: 40
// bytes of shared scratch for the sample; pi: the rollout's chase store;
// ring: a history ring to continue (a copy of the root's is made), or
// nullptr to keep no history (the last two moves come from the root's).
// Returns the tally slot: 0 win, 1 loss, 2 draw for the player to move at
// the root, 3 unfinished.
template <int L>
__device__ __forceinline__ int rollout_one(SmemGame* G, uint8_t* types_s, uint64_t* pi, uint16_t* ring,
                                           const Team<L>& T, const RootState* R, const BeliefPlan* plan,
                                           const uint8_t* types, int depth, uint32_t k0, uint32_t k1, uint32_t stream,
                                           uint32_t k, const Rules& Rl)
{
    begin_rollout(G, types_s, pi, ring, T, R, plan, types, k0, k1, stream, k);
    const int searcher = G->c.ply & 1;
    int n = gen_moves(G, T, searcher, Rl.flags, false, true, pi, (uint32_t*)nullptr);
    int code = 0, winner = -1;
    if (n == 0) start_end(G, T, Rl, pi, code, winner);
    for (int d = 0; !code && d < depth; ++d) {
        const uint4 w = philox(make_uint4(stream, k, (uint32_t)d, 4u << 24), k0, k1);
        if (Rl.flags & kMagnet) magnet_apply(G, T, w.x, w.y, ring, pi, Rl.flags);
        else select_apply(G, T, -1, uniform_below(w.x, (uint32_t)n), ring, pi, Rl.flags);
        check_end(G, T, Rl, pi, code, winner, n, (uint32_t*)nullptr);
    }
    return tally_slot(code, winner, searcher);
}

// Team: one rollout of the per-move search (App. E "Search", step 2) from
// root R: belief sample `s` of R's plan (given in `types`, or drawn), the
// searcher's move `first` (legal
// at the root, whatever the sample), then up to depth-1 plies of the rollout
// policy, ply d drawing from Philox at counter (stream, c1, d, 5<<24) with
// c1 = j*S+s.
// No history ring is kept.  Returns the tally slot as rollout_one does.
template <int L>
__device__ __forceinline__ int search_rollout(SmemGame* G, uint8_t* types_s, uint64_t* pi, const Team<L>& T,
                                              const RootState* R, const uint8_t* types, int first, int depth,
                                              uint32_t k0, uint32_t k1, uint32_t stream, uint32_t c1, uint32_t s,
                                              const Rules& Rl)
{
    begin_rollout(G, types_s, pi, (uint16_t*)nullptr, T, R, &R->plan, types, k0, k1, stream, s);
    // the root's side to move, from the root record (the game record's ply
    // changes when the forced first move is played)
    const int searcher = R->c.ply & 1;
    int code = 0, winner = -1, n = 0;
    select_apply(G, T, first, 0u, (uint16_t*)nullptr, pi, Rl.flags);
    check_end(G, T, Rl, pi, code, winner, n, (uint32_t*)nullptr);
    for (int d = 1; !code && d < depth; ++d) {
        const uint4 w = philox(make_uint4(stream, c1, (uint32_t)d, 5u << 24), k0, k1);
        if (Rl.flags & kMagnet) magnet_apply(G, T, w.x, w.y, (uint16_t*)nullptr, pi, Rl.flags);
        else select_apply(G, T, -1, uniform_below(w.x, (uint32_t)n), (uint16_t*)nullptr, pi, Rl.flags);
        check_end(G, T, Rl, pi, code, winner, n, (uint32_t*)nullptr);
    }
    return tally_slot(code, winner, searcher);
}

}  // namespace stg
