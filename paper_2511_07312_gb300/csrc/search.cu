// search.cu -- belief samples of the opponent's hidden pieces and random
// rollouts from each sample (App. E "Search", steps 1-2, with the uniform
// posterior over consistent assignments in place of the belief network and a
// uniform random policy in place of the move network).
//
// k_belief: one block per position; the position is read once into shared
// memory, its hidden-piece lists and remaining counts are built once, and
// every lane then draws whole samples (Fisher-Yates over at most 40 slots)
// with its own Philox stream.
// k_rollout: one block per position; each warp copies the shared root state,
// substitutes one sample's types and plays the rollout with the warp engine,
// tallies reduced in shared memory.
#include "engine.cuh"
#include "snapshot.cuh"
#include "host_common.h"

using namespace stg;

namespace {

// Hidden-piece structure of one position, from the searching player's view.
struct __align__(16) BeliefPlan {
    uint8_t known[40];      // type of opponent piece i if public, else 0xFF
    uint8_t order[40];      // hidden pieces in ascending square order
    uint8_t is_unmoved[40]; // per entry of order
    uint8_t movable[40];    // sorted movable multiset still to place
    int n_hidden, n_unmoved, n_flag, n_imm, n_mov;
    int opp;
};

__device__ void make_plan(const SmemGame* G, BeliefPlan* B)
{
    // single thread
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

// One sample (single thread): the types of opponent pieces 0..39.
__device__ void draw_sample(const BeliefPlan* B, uint32_t k0, uint32_t k1, uint32_t stream, uint32_t sample,
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
    // 1. immovable pieces onto n_imm of the unmoved hidden pieces
    uint8_t idx[40], imm[40];
    const int nu = B->n_unmoved;
    for (int i = 0; i < nu; ++i) { idx[i] = (uint8_t)i; imm[i] = 0xFF; }
    for (int i = 0; i < B->n_imm && i < nu; ++i) {
        const int j = i + (int)uniform_below(next(), (uint32_t)(nu - i));
        const uint8_t t = idx[i]; idx[i] = idx[j]; idx[j] = t;
        imm[idx[i]] = (uint8_t)(i < B->n_flag ? kFlag : kBomb);
    }
    // 2. the movable multiset over the remaining hidden pieces
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

struct __align__(16) RootSmem {
    SmemGame g;
    uint64_t pi[kPiCap];
    uint16_t ring[kRing];
    BeliefPlan plan;
    int bad;
};

struct __align__(16) WarpSmem {
    SmemGame g;
    uint64_t pi[kPiCap];
    uint16_t ring[kRing];
    uint8_t types[40];
};

__device__ int load_root(RootSmem* R, const st_position* pos)
{
    // warp 0 imports; the block waits
    if (threadIdx.x < 32) {
        const int bad = import_position(&R->g, pos, R->ring, R->pi);
        if (threadIdx.x == 0) {
            R->bad = bad;
            if (!bad) make_plan(&R->g, &R->plan);
        }
    }
    __syncthreads();
    return R->bad;
}

__global__ void k_belief(const st_position* pos, int P, int K, uint32_t k0, uint32_t k1, const uint32_t* stream_ids,
                         uint8_t* types, uint8_t* status)
{
    __shared__ RootSmem R;
    const int p = blockIdx.x;
    if (p >= P) return;
    const int bad = load_root(&R, pos + p);
    if (threadIdx.x == 0 && status) status[p] = bad ? 1 : 0;
    uint8_t* out = types + (size_t)p * K * 40;
    if (bad) {
        for (int i = threadIdx.x; i < K * 40; i += blockDim.x) out[i] = 0;
        return;
    }
    const uint32_t stream = stream_ids ? stream_ids[p] : (uint32_t)p;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        uint8_t t[40];
        draw_sample(&R.plan, k0, k1, stream, (uint32_t)k, t);
        uint32_t* o = reinterpret_cast<uint32_t*>(out + (size_t)k * 40);
        for (int i = 0; i < 10; ++i)
            o[i] = (uint32_t)t[4 * i] | ((uint32_t)t[4 * i + 1] << 8) | ((uint32_t)t[4 * i + 2] << 16) |
                   ((uint32_t)t[4 * i + 3] << 24);
    }
}

constexpr int kRolloutWarps = 8;

__global__ void k_rollout(const st_position* pos, int P, int K, int depth, uint32_t k0, uint32_t k1,
                          const uint32_t* stream_ids, const uint8_t* types_in, Rules Rl, int32_t* tallies,
                          uint8_t* status)
{
    __shared__ RootSmem R;
    __shared__ int tl[4];
    extern __shared__ __align__(16) unsigned char smem[];
    WarpSmem* W = reinterpret_cast<WarpSmem*>(smem) + (threadIdx.x >> 5);
    const int p = blockIdx.x;
    if (p >= P) return;
    if (threadIdx.x < 4) tl[threadIdx.x] = 0;
    const int bad = load_root(&R, pos + p);
    if (threadIdx.x == 0 && status) status[p] = bad ? 1 : 0;
    if (bad) {
        if (threadIdx.x < 4) tallies[4 * (size_t)p + threadIdx.x] = 0;
        return;
    }
    const int lane = lane_id();
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const uint32_t stream = stream_ids ? stream_ids[p] : (uint32_t)p;
    const int searcher = R.g.c.ply & 1, opp = 1 - searcher;
    const int npi = R.g.c.n_pi;
    SmemGame* G = &W->g;
    for (int k = warp; k < K; k += nwarps) {
        {
            const uint4* src = reinterpret_cast<const uint4*>(&R.g);
            uint4* dst = reinterpret_cast<uint4*>(G);
            for (int i = lane; i < (int)(sizeof(SmemGame) / 16); i += 32) dst[i] = src[i];
            const uint4* rs = reinterpret_cast<const uint4*>(R.ring);
            uint4* rd = reinterpret_cast<uint4*>(W->ring);
            for (int i = lane; i < kRing * 2 / 16; i += 32) rd[i] = rs[i];
            for (int i = lane; i < npi; i += 32) W->pi[i] = R.pi[i];
        }
        if (types_in) {
            const uint8_t* t = types_in + ((size_t)p * K + k) * 40;
            for (int i = lane; i < 40; i += 32) W->types[i] = t[i];
            if (lane < 8) W->types[32 + lane] = t[32 + lane];
        } else if (lane == 0) {
            draw_sample(&R.plan, k0, k1, stream, (uint32_t)k, W->types);
        }
        __syncwarp();
        for (int i = lane; i < 40; i += 32) G->c.type[opp * 40 + i] = W->types[i];
        if (lane < 8) G->c.type[opp * 40 + 32 + lane] = W->types[32 + lane];
        __syncwarp();
        int n = gen_moves(G, searcher, Rl.flags, false, true, W->ring, W->pi);
        int code = 0, winner = -1;
        if (n == 0) start_end(G, Rl, W->ring, W->pi, code, winner);
        for (int d = 0; !code && d < depth; ++d) {
            const uint4 w = philox(make_uint4(stream, (uint32_t)k, (uint32_t)d, 4u << 24), k0, k1);
            const int a = select_action(G, uniform_below(w.x, (uint32_t)n));
            apply_move(G, a, W->ring, W->pi);
            check_end(G, Rl, W->ring, W->pi, code, winner, n);
        }
        if (lane == 0) {
            const int slot = !code ? 3 : (winner < 0 ? 2 : (winner == searcher ? 0 : 1));
            atomicAdd(&tl[slot], 1);
        }
        __syncwarp();
    }
    __syncthreads();
    if (threadIdx.x < 4) tallies[4 * (size_t)p + threadIdx.x] = tl[threadIdx.x];
}

}  // namespace

extern "C" st_status st_belief_sample(const st_position* pos, int32_t P, int32_t K, uint64_t seed,
                                      const uint32_t* stream_ids, uint8_t* types, uint8_t* item_status, void* stream)
{
    ST_CHECK_ARG(P >= 0 && K >= 0, "st_belief_sample: negative size");
    if (P == 0 || K == 0) return ST_OK;
    ST_CHECK_ARG(pos && types, "st_belief_sample: null argument");
    ST_CHECK_ARG(((uintptr_t)types & 3u) == 0, "st_belief_sample: types must be 4-byte aligned");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    k_belief<<<P, 128, 0, s>>>(pos, P, K, (uint32_t)seed, (uint32_t)(seed >> 32), stream_ids, types, item_status);
    ST_CUDA(cudaGetLastError());
    return ST_OK;
}

extern "C" st_status st_rollout(const st_position* pos, int32_t P, int32_t K, int32_t depth, uint64_t seed,
                                const uint32_t* stream_ids, const uint8_t* types, const st_rules* rules,
                                int32_t* tallies, uint8_t* item_status, void* stream)
{
    ST_CHECK_ARG(rules_ok(rules), "st_rollout: invalid rules");
    ST_CHECK_ARG(P >= 0 && K >= 0 && depth >= 0, "st_rollout: negative size");
    if (P == 0) return ST_OK;
    ST_CHECK_ARG(pos && tallies, "st_rollout: null argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Rules r;
    r.k = rules->battleless_limit;
    r.cap = rules->max_plies;
    r.flags = rules->flags;
    k_rollout<<<P, 32 * kRolloutWarps, kRolloutWarps * sizeof(WarpSmem), s>>>(
        pos, P, K, depth, (uint32_t)seed, (uint32_t)(seed >> 32), stream_ids, types, r, tallies, item_status);
    ST_CUDA(cudaGetLastError());
    return ST_OK;
}
