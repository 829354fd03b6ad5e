// search.cu -- belief samples of the opponent's hidden pieces, rollouts from
// each sample, and the per-move search with its policy update (App. E
// "Search", steps 1-4, with the uniform posterior over consistent
// assignments in place of the belief network and the uniform or magnet
// rollout policy in place of the move network).
//
// k_belief: one block per position; the position is read once into shared
// memory, its hidden-piece plan is built once, and every thread then draws
// whole samples (Fisher-Yates over at most 40 pieces) from its own Philox
// stream.
// st_rollout: k_roots imports every position once (one warp each) into a
// root record in HBM; k_draw_samples draws every belief sample ahead (a
// thread per sample); k_rollout_flat runs one 4-lane team per (position,
// sample) at a time on a resident grid, copying the root into shared memory,
// so a single position's samples spread over the whole GPU.  A rollout keeps
// no history ring (its last two moves start from the root's) and its chase
// store sits in a global scratch slot of its team.
// st_positions_mask: legal masks of snapshots (App. B.1 ComputeLegalActionMask).
// st_search (steps 1-4): k_search_prep imports every position, lists the
// searcher's legal moves in ascending order and clears the outputs;
// k_search_offsets turns the move counts into unit offsets; k_draw_samples
// draws each configuration once; k_search_rollouts runs one 4-lane team per
// (position, move, sample) unit at a time on a resident grid; k_search_policy
// forms the values, the magnet policy, the update and the sampled move, one
// warp per position.
#include <algorithm>
#include <atomic>
#include <math_constants.h>
#include "rollout.cuh"
#include "host_common.h"

using namespace stg;

namespace {

struct __align__(16) BeliefSmem {
    SmemGame g;
    uint64_t pi[kPiWords];
    uint16_t ring[kRing];
    BeliefPlan plan;
    int bad;
};

__global__ void k_belief(const st_position* pos, int P, int K, uint32_t k0, uint32_t k1, const uint32_t* stream_ids,
                         uint8_t* types, uint8_t* status)
{
    __shared__ BeliefSmem R;
    const int p = blockIdx.x;
    if (p >= P) return;
    if (threadIdx.x < 32) {
        const int bad = import_position(&R.g, pos + p, R.ring, R.pi);
        if (threadIdx.x == 0) {
            R.bad = bad;
            if (!bad) make_plan(&R.g, &R.plan);
        }
    }
    __syncthreads();
    const int bad = R.bad;
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

constexpr int kRootWarps = 4;
constexpr int kFlatLanes = 4;                              // one rollout per 4-lane team
constexpr int kFlatWarps = 2;
constexpr int kFlatTeams = 32 * kFlatWarps / kFlatLanes;   // rollouts per block
constexpr int kFlatMinBlocks = 12;                          // resident blocks per SM the registers allow

__global__ void k_roots(const st_position* pos, int P, RootState* roots, uint8_t* status)
{
    extern __shared__ __align__(16) unsigned char smem[];
    RolloutSmem* S = reinterpret_cast<RolloutSmem*>(smem) + (threadIdx.x >> 5);
    const int p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (p >= P) return;
    build_root(S, pos + p, roots + p);
    if (lane_id() == 0 && status) status[p] = roots[p].bad ? 1 : 0;
}

// Thread per (position, sample): sample k of position p's plan into
// types[p*K + k][40] (App. E step 1), so that rollout teams only read their
// sample.  Consecutive threads share a position, whose plan comes from L1.
__global__ void k_draw_samples(const RootState* roots, int P, int K, uint32_t k0, uint32_t k1,
                               const uint32_t* stream_ids, uint8_t* types)
{
    const long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= (long long)P * K) return;
    const int p = (int)(u / K), k = (int)(u - (long long)p * K);
    const RootState* R = roots + p;
    if (R->bad) return;
    const uint32_t stream = stream_ids ? stream_ids[p] : (uint32_t)p;
    uint8_t t[40];
    draw_sample(&R->plan, k0, k1, stream, (uint32_t)k, t);
    uint2* o = reinterpret_cast<uint2*>(types + (size_t)u * 40);
    for (int i = 0; i < 5; ++i) {
        const uint8_t* b = t + 8 * i;
        o[i] = make_uint2((uint32_t)b[0] | ((uint32_t)b[1] << 8) | ((uint32_t)b[2] << 16) | ((uint32_t)b[3] << 24),
                          (uint32_t)b[4] | ((uint32_t)b[5] << 8) | ((uint32_t)b[6] << 16) | ((uint32_t)b[7] << 24));
    }
}

// Samples are drawn ahead of the rollouts for calls of at least this many
// rollouts (below it the extra launch and allocation cost more than the
// draws they save) while they fit this many bytes.
constexpr long long kDrawAheadMinUnits = 16384;
constexpr size_t kDrawAheadBytes = (size_t)1 << 30;

// One (position, sample) unit per 4-lane team at a time, grid-stride over
// the units with a grid of resident blocks; consecutive teams of a block
// share a position, so its root and plan come mostly from L1.  A rollout
// keeps no history ring (its last two moves start from the root's); its
// chase store is the team's slot of pi_scratch.
__global__ void __launch_bounds__(32 * kFlatWarps, kFlatMinBlocks) k_rollout_flat(const RootState* roots, int P, int K, int depth, uint32_t k0, uint32_t k1,
                               const uint32_t* stream_ids, const uint8_t* types_in, Rules Rl, int32_t* tallies,
                               uint64_t* pi_scratch)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const Team<kFlatLanes> T;
    const int team = threadIdx.x / kFlatLanes;
    FlatSmem* S = reinterpret_cast<FlatSmem*>(smem) + team;
    uint64_t* pi = pi_scratch + ((size_t)blockIdx.x * kFlatTeams + team) * kPiWords;
    if (K <= 0) return;
    // unit u = p*K + k, this team's units u0, u0 + stride, ...: (p, k) is
    // stepped by the stride's quotient and remainder instead of dividing
    // each unit (no 64-bit counter held across the rollout)
    const long long u0 = (long long)blockIdx.x * kFlatTeams + team;
    const long long stride = (long long)gridDim.x * kFlatTeams;
    int p = (int)(u0 / K), k = (int)(u0 - (long long)p * K);
    const int dp = (int)(stride / K), dk = (int)(stride - (long long)dp * K);
    for (; p < P; p += dp, k += dk, p += k >= K ? 1 : 0, k -= k >= K ? K : 0) {
        const RootState* R = roots + p;
        if (R->bad) continue;
        const uint32_t stream = stream_ids ? stream_ids[p] : (uint32_t)p;
        const uint8_t* t = types_in ? types_in + ((size_t)p * K + k) * 40 : nullptr;
        const int out = rollout_one(&S->g, S->types, pi, (uint16_t*)nullptr, T, R, &R->plan, t, depth, k0, k1,
                                    stream, (uint32_t)k, Rl);
        if (T.leader()) atomicAdd(&tallies[4 * (size_t)p + out], 1);
        T.sync();
    }
}

// Resident blocks per SM of the rollout kernels (both share the shape).
int flat_blocks_per_sm()
{
    static std::atomic<int> cached[64];   // 0 until looked up (threads may race to fill a slot; same value)
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    int occ = cached[dev].load(std::memory_order_relaxed);
    if (!occ) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_rollout_flat, 32 * kFlatWarps,
                                                          kFlatTeams * sizeof(FlatSmem)) != cudaSuccess || occ < 1) {
            cudaGetLastError();
            occ = 1;
        }
        cached[dev].store(occ, std::memory_order_relaxed);
    }
    return occ;
}

// ----------------------------------------------------------------- st_search
constexpr int kSearchMoves = ST_SEARCH_MAX_MOVES;
constexpr int kMaskWordsUsed = (10000 + 31) / 32;                  // 313
constexpr int kCompactWords = (kMaskWordsUsed + 31) / 32;          // mask words per lane

// Warp per position: root record, the searcher's legal moves ascending, and
// every output of the position cleared.
__global__ void k_search_prep(const st_position* pos, int P, Rules Rl, RootState* roots, int32_t* n_moves,
                              int16_t* actions, int32_t* tallies, double* q, double* pi, int16_t* chosen,
                              uint8_t* status)
{
    extern __shared__ __align__(16) unsigned char smem[];
    RolloutSmem* S = reinterpret_cast<RolloutSmem*>(smem) + (threadIdx.x >> 5);
    const int p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (p >= P) return;
    const Team<32> T;
    const int lane = T.tl;
    int16_t* act = actions + (size_t)p * kSearchMoves;
    {
        int4* tl = reinterpret_cast<int4*>(tallies + (size_t)p * kSearchMoves * 4);
        for (int i = lane; i < kSearchMoves; i += 32) {
            tl[i] = make_int4(0, 0, 0, 0);
            q[(size_t)p * kSearchMoves + i] = 0.0;
            pi[(size_t)p * kSearchMoves + i] = 0.0;
        }
    }
    int bad_w = build_root(S, pos + p, roots + p);
    int n = 0;
    uint32_t words[kCompactWords];
    int mine = 0;
    if (!bad_w) {
        n = gen_moves(&S->g, T, S->g.c.ply & 1, Rl.flags, false, true, S->pi, S->mask);
        if (n > kSearchMoves) { bad_w = 14; n = 0; }   // more moves than a position can have
        for (int i = 0; i < kCompactWords; ++i) {
            const int w = lane * kCompactWords + i;
            words[i] = w < kMaskWordsUsed ? S->mask[w] : 0u;
            mine += __popc(words[i]);
        }
    }
    uint32_t before = mine;
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t v = T.shfl_up(before, d);
        if (lane >= d) before += v;
    }
    before -= mine;   // moves listed by lower lanes
    for (int i = lane; i < kSearchMoves; i += 32)
        if (i >= n) act[i] = -1;
    if (!bad_w) {
        int o = (int)before;
        for (int i = 0; i < kCompactWords; ++i) {
            uint32_t m = words[i];
            const int base = 32 * (lane * kCompactWords + i);
            while (m) {
                const int b = __ffs(m) - 1;
                m &= m - 1;
                act[o++] = (int16_t)(base + b);
            }
        }
    }
    if (lane == 0) {
        n_moves[p] = bad_w ? 0 : n;
        chosen[p] = -1;
        if (status) status[p] = bad_w ? 1 : 0;
    }
}

// Single block: offs[p] = S * (moves of positions before p), offs[P] = total.
constexpr int kOffsetThreads = 1024;

__global__ void __launch_bounds__(kOffsetThreads) k_search_offsets(const int32_t* n_moves, int P, int S,
                                                                   long long* offs)
{
    __shared__ long long part[kOffsetThreads];
    const int per = (P + kOffsetThreads - 1) / kOffsetThreads;
    const int a = threadIdx.x * per, b = min(P, a + per);
    long long sum = 0;
    for (int i = a; i < b; ++i) sum += (long long)n_moves[i] * S;
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int d = 1; d < kOffsetThreads; d <<= 1) {
        const long long v = threadIdx.x >= d ? part[threadIdx.x - d] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    long long run = part[threadIdx.x] - sum;
    for (int i = a; i < b; ++i) {
        offs[i] = run;
        run += (long long)n_moves[i] * S;
    }
    if (threadIdx.x == kOffsetThreads - 1) offs[P] = part[threadIdx.x];
}

// One (position, move j, sample s) unit per 4-lane team, unit u of position
// p being offs[p] + j*S + s; consecutive teams share a position and mostly a
// move.  Grid-stride over the units.
__global__ void __launch_bounds__(32 * kFlatWarps, kFlatMinBlocks) k_search_rollouts(const RootState* roots, const long long* offs, int P, int S, int depth, uint32_t k0,
                                  uint32_t k1, const uint32_t* stream_ids, const int16_t* actions, Rules Rl,
                                  int32_t* tallies, uint64_t* pi_scratch, const uint8_t* types)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const Team<kFlatLanes> T;
    FlatSmem* F = reinterpret_cast<FlatSmem*>(smem) + threadIdx.x / kFlatLanes;
    uint64_t* pi = pi_scratch + ((size_t)blockIdx.x * kFlatTeams + threadIdx.x / kFlatLanes) * kPiWords;
    const long long total = offs[P];
    const long long stride = (long long)gridDim.x * kFlatTeams;
    for (long long u = (long long)blockIdx.x * kFlatTeams + threadIdx.x / kFlatLanes; u < total; u += stride) {
        int lo = 0, hi = P;   // the last p with offs[p] <= u
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (offs[mid] <= u) lo = mid;
            else hi = mid;
        }
        const int p = lo;
        const int r = (int)(u - offs[p]);
        const int j = r / S, s = r - j * S;
        const RootState* R = roots + p;
        const uint32_t stream = stream_ids ? stream_ids[p] : (uint32_t)p;
        const int first = actions[(size_t)p * kSearchMoves + j];
        const uint8_t* ty = types ? types + ((size_t)p * S + s) * 40 : nullptr;
        const int out = search_rollout(&F->g, F->types, pi, T, R, ty, first, depth, k0, k1, stream, (uint32_t)r,
                                       (uint32_t)s, Rl);
        if (T.leader()) atomicAdd(&tallies[((size_t)p * kSearchMoves + j) * 4 + out], 1);
        T.sync();
    }
}

constexpr int kPolicyWarps = 4;

// Warp per position: q, rho, the update in double and the sampled move.
// Products, sums and quotients are rounded one at a time in the order the
// update is written (no contraction), so only log and exp differ from a
// correctly rounded evaluation, by at most an ulp or two.
__global__ void k_search_policy(int P, int S, uint32_t k0, uint32_t k1, const uint32_t* stream_ids,
                                const float* pi_theta, const float* q_values, double alpha, double beta,
                                const int32_t* n_moves,
                                const int16_t* actions, const int32_t* tallies, double* q, double* pi, int16_t* chosen,
                                uint8_t* status)
{
    __shared__ double wsh[kPolicyWarps][kSearchMoves];
    const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p = blockIdx.x * kPolicyWarps + wi;
    if (p >= P) return;
    const int n = n_moves[p];
    if (n == 0) return;
    const int16_t* act = actions + (size_t)p * kSearchMoves;
    double* qp = q + (size_t)p * kSearchMoves;
    double* pp = pi + (size_t)p * kSearchMoves;
    double* w = wsh[wi];
    // pieces with a legal move: runs of equal from-squares in the ascending list
    int starts = 0;
    for (int j = lane; j < n; j += 32) starts += (j == 0 || act[j] / 100 != act[j - 1] / 100);
    const int pieces = __reduce_add_sync(0xffffffffu, (unsigned)starts);
    const double ab = __dadd_rn(alpha, beta);
    double zmax = -CUDART_INF;
    for (int j = lane; j < n; j += 32) {
        const int a = act[j], f = a / 100;
        double qj;
        if (q_values) {
            qj = (double)q_values[(size_t)p * 10000 + a];
        } else {
            const int4 t = reinterpret_cast<const int4*>(tallies + (size_t)p * kSearchMoves * 4)[j];
            qj = S > 0 ? __ddiv_rn((double)(t.x - t.y), (double)S) : 0.0;
        }
        qp[j] = qj;
        int lo = j, hi = j;
        while (lo > 0 && act[lo - 1] / 100 == f) --lo;
        while (hi + 1 < n && act[hi + 1] / 100 == f) ++hi;
        const double rho = __ddiv_rn(1.0, __dmul_rn((double)pieces, (double)(hi - lo + 1)));
        const double pt = pi_theta ? (double)pi_theta[(size_t)p * 10000 + a] : __ddiv_rn(1.0, (double)n);
        double z = -CUDART_INF;
        if (pt > 0.0)
            z = __ddiv_rn(__dadd_rn(__dadd_rn(qj, __dmul_rn(alpha, log(rho))), __dmul_rn(beta, log(pt))), ab);
        w[j] = z;
        zmax = fmax(zmax, z);
    }
    for (int d = 16; d >= 1; d >>= 1) zmax = fmax(zmax, __shfl_xor_sync(0xffffffffu, zmax, d));
    if (zmax == -CUDART_INF) {
        if (lane == 0 && status) status[p] = 2;
        return;
    }
    for (int j = lane; j < n; j += 32) w[j] = w[j] == -CUDART_INF ? 0.0 : exp(__dadd_rn(w[j], -zmax));
    __syncwarp();
    double W = 0.0;
    if (lane == 0) {
        for (int j = 0; j < n; ++j) W = __dadd_rn(W, w[j]);
        const uint32_t stream = stream_ids ? stream_ids[p] : (uint32_t)p;
        const uint4 r = philox(make_uint4(stream, 0u, 0u, 6u << 24), k0, k1);
        const double u = ((double)(r.x >> 5) * 67108864.0 + (double)(r.y >> 6)) / 9007199254740992.0;   // exact
        const double t = __dmul_rn(u, W);
        double c = 0.0;
        int pick = n - 1;
        for (int j = 0; j < n; ++j) {
            c = __dadd_rn(c, w[j]);
            if (t < c) { pick = j; break; }
        }
        chosen[p] = act[pick];
    }
    W = __shfl_sync(0xffffffffu, W, 0);
    for (int j = lane; j < n; j += 32) pp[j] = __ddiv_rn(w[j], W);
}

// Warp per snapshot: the legal mask of the player to move, its move count,
// and whether the two-square rule removes one of its moves.
__global__ void k_positions_mask(const st_position* pos, int P, Rules Rl, uint8_t* mask, int32_t* n_legal,
                                 uint8_t* two_square, uint8_t* status)
{
    extern __shared__ __align__(16) unsigned char smem[];
    RolloutSmem* S = reinterpret_cast<RolloutSmem*>(smem) + (threadIdx.x >> 5);
    const int p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (p >= P) return;
    const Team<32> T;
    const int lane = T.tl;
    const int bad = import_position(&S->g, pos + p, S->ring, S->pi);
    int n = 0, ts = 0;
    if (!bad) {
        const int Pl = S->g.c.ply & 1;
        n = gen_moves(&S->g, T, Pl, Rl.flags, false, true, S->pi,
                      mask ? reinterpret_cast<uint32_t*>(mask + (size_t)p * kMaskBytes) : nullptr);
        if (Rl.flags & kTwoSquare) {
            const int n_ts = gen_moves(&S->g, T, Pl, kTwoSquare, false, false, S->pi, (uint32_t*)nullptr);
            const int n_ph = gen_moves(&S->g, T, Pl, 0u, true, false, S->pi, (uint32_t*)nullptr);
            ts = n_ts < n_ph;
        }
    } else if (mask) {
        uint4* d = reinterpret_cast<uint4*>(mask + (size_t)p * kMaskBytes);
        for (int i = lane; i < kMaskBytes / 16; i += 32) d[i] = make_uint4(0, 0, 0, 0);
    }
    if (lane == 0) {
        if (n_legal) n_legal[p] = n;
        if (two_square) two_square[p] = (uint8_t)ts;
        if (status) status[p] = bad ? 1 : 0;
    }
}

}  // namespace

extern "C" st_status st_belief_sample(const st_position* pos, int32_t P, int32_t K, uint64_t seed,
                                      const uint32_t* stream_ids, uint8_t* types, uint8_t* item_status, void* stream)
{
    ST_NVTX("st_belief_sample");
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
    ST_NVTX("st_rollout");
    ST_CHECK_ARG(rules_ok(rules, true), "st_rollout: invalid rules");
    ST_CHECK_ARG(P >= 0 && K >= 0 && depth >= 0, "st_rollout: negative size");
    if (P == 0) return ST_OK;
    ST_CHECK_ARG(pos && tallies, "st_rollout: null argument");
    ST_CHECK_ARG((long long)P * K < (1LL << 40), "st_rollout: P*K too large");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Rules r;
    r.k = rules->battleless_limit;
    r.cap = rules->max_plies;
    r.flags = rules->flags;
    RootState* roots = nullptr;
    ST_CUDA(cudaMallocAsync(&roots, (size_t)P * sizeof(RootState), s));
    cudaError_t err = cudaMemsetAsync(tallies, 0, (size_t)P * 4 * sizeof(int32_t), s);
    if (err == cudaSuccess) {
        const int rb = (P + kRootWarps - 1) / kRootWarps;
        k_roots<<<rb, 32 * kRootWarps, kRootWarps * sizeof(RolloutSmem), s>>>(pos, P, roots, item_status);
        err = cudaGetLastError();
    }
    uint64_t* pi_scratch = nullptr;
    uint8_t* drawn = nullptr;
    if (err == cudaSuccess && K > 0) {
        const long long units = (long long)P * K;
        const long long fb = std::min((units + kFlatTeams - 1) / kFlatTeams,
                                      (long long)sm_count() * flat_blocks_per_sm());
        err = cudaMallocAsync(&pi_scratch, (size_t)fb * kFlatTeams * kPiWords * sizeof(uint64_t), s);
        // without given samples, draw them ahead in one wide launch when they fit
        const uint8_t* ty = types;
        if (err == cudaSuccess && !types && units >= kDrawAheadMinUnits && (size_t)units * 40 <= kDrawAheadBytes &&
            cudaMallocAsync(&drawn, (size_t)units * 40, s) == cudaSuccess) {
            k_draw_samples<<<(unsigned)((units + 127) / 128), 128, 0, s>>>(roots, P, K, (uint32_t)seed,
                                                                          (uint32_t)(seed >> 32), stream_ids, drawn);
            err = cudaGetLastError();
            ty = drawn;
        }
        cudaGetLastError();   // a failed draw-ahead allocation leaves the in-kernel draw
        if (err == cudaSuccess) {
            k_rollout_flat<<<(unsigned)fb, 32 * kFlatWarps, kFlatTeams * sizeof(FlatSmem), s>>>(
                roots, P, K, depth, (uint32_t)seed, (uint32_t)(seed >> 32), stream_ids, ty, r, tallies,
                pi_scratch);
            err = cudaGetLastError();
        }
    }
    if (drawn) cudaFreeAsync(drawn, s);
    if (pi_scratch) cudaFreeAsync(pi_scratch, s);
    cudaFreeAsync(roots, s);
    if (err != cudaSuccess) {
        stg::set_error("st_rollout: launch failed: %s", cudaGetErrorString(err));
        return ST_ERR_CUDA;
    }
    return ST_OK;
}

extern "C" st_status st_search(const st_position* pos, int32_t P, int32_t S, int32_t depth, uint64_t seed,
                               const uint32_t* stream_ids, const float* pi_theta, const float* q_values,
                               double alpha, double beta,
                               const st_rules* rules, int32_t* n_moves, int16_t* actions, int32_t* tallies,
                               double* q, double* pi, int16_t* chosen, uint8_t* item_status, void* stream)
{
    ST_NVTX("st_search");
    ST_CHECK_ARG(rules_ok(rules, true), "st_search: invalid rules");
    ST_CHECK_ARG(P >= 0 && P <= 65535, "st_search: P must be in [0, 65535]");
    ST_CHECK_ARG(S >= 0 && S <= (1 << 24), "st_search: S must be in [0, 2^24]");
    ST_CHECK_ARG(depth >= 1, "st_search: depth must be >= 1");
    ST_CHECK_ARG(alpha >= 0.0 && beta >= 0.0 && alpha + beta > 0.0 && alpha + beta < 1e300,
                 "st_search: alpha, beta must be finite, >= 0, with a positive sum");
    if (P == 0) return ST_OK;
    ST_CHECK_ARG(pos && n_moves && actions && tallies && q && pi && chosen, "st_search: null argument");
    ST_CHECK_ARG(aligned16(tallies), "st_search: tallies must be 16-byte aligned");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Rules r;
    r.k = rules->battleless_limit;
    r.cap = rules->max_plies;
    r.flags = rules->flags;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    RootState* roots = nullptr;
    long long* offs = nullptr;
    ST_CUDA(cudaMallocAsync(&roots, (size_t)P * sizeof(RootState), s));
    cudaError_t err = cudaMallocAsync(&offs, (size_t)(P + 1) * sizeof(long long), s);
    if (err == cudaSuccess) {
        const int rb = (P + kRootWarps - 1) / kRootWarps;
        k_search_prep<<<rb, 32 * kRootWarps, kRootWarps * sizeof(RolloutSmem), s>>>(
            pos, P, r, roots, n_moves, actions, tallies, q, pi, chosen, item_status);
        err = cudaGetLastError();
    }
    if (err == cudaSuccess && S > 0 && !q_values) {
        k_search_offsets<<<1, kOffsetThreads, 0, s>>>(n_moves, P, S, offs);
        err = cudaGetLastError();
        if (err == cudaSuccess) {
            // at most 244 moves per position; grid-stride beyond 2^24 blocks
            const long long units = (long long)P * 244 * S;
            const long long fb = std::min((units + kFlatTeams - 1) / kFlatTeams,
                                          (long long)sm_count() * flat_blocks_per_sm());
            uint64_t* pi_scratch = nullptr;
            uint8_t* drawn = nullptr;
            err = cudaMallocAsync(&pi_scratch, (size_t)fb * kFlatTeams * kPiWords * sizeof(uint64_t), s);
            // configuration s of position p serves every move: drawn once, ahead
            const long long samples = (long long)P * S;
            if (err == cudaSuccess && (size_t)samples * 40 <= kDrawAheadBytes &&
                cudaMallocAsync(&drawn, (size_t)samples * 40, s) == cudaSuccess) {
                k_draw_samples<<<(unsigned)((samples + 127) / 128), 128, 0, s>>>(roots, P, S, k0, k1, stream_ids,
                                                                                drawn);
                err = cudaGetLastError();
            }
            cudaGetLastError();   // a failed draw-ahead allocation leaves the in-kernel draw
            if (err == cudaSuccess) {
                k_search_rollouts<<<(unsigned)fb, 32 * kFlatWarps, kFlatTeams * sizeof(FlatSmem), s>>>(
                    roots, offs, P, S, depth, k0, k1, stream_ids, actions, r, tallies, pi_scratch, drawn);
                err = cudaGetLastError();
            }
            if (drawn) cudaFreeAsync(drawn, s);
            if (pi_scratch) cudaFreeAsync(pi_scratch, s);
        }
    }
    if (err == cudaSuccess) {
        k_search_policy<<<(P + kPolicyWarps - 1) / kPolicyWarps, 32 * kPolicyWarps, 0, s>>>(
            P, S, k0, k1, stream_ids, pi_theta, q_values, alpha, beta, n_moves, actions, tallies, q, pi, chosen,
            item_status);
        err = cudaGetLastError();
    }
    if (offs) cudaFreeAsync(offs, s);
    cudaFreeAsync(roots, s);
    if (err != cudaSuccess) {
        stg::set_error("st_search: launch failed: %s", cudaGetErrorString(err));
        return ST_ERR_CUDA;
    }
    return ST_OK;
}

extern "C" st_status st_positions_mask(const st_position* pos, int32_t P, const st_rules* rules, uint8_t* mask,
                                       int32_t* n_legal, uint8_t* two_square, uint8_t* item_status, void* stream)
{
    ST_NVTX("st_positions_mask");
    ST_CHECK_ARG(rules_ok(rules), "st_positions_mask: invalid rules");
    ST_CHECK_ARG(P >= 0, "st_positions_mask: P < 0");
    if (P == 0) return ST_OK;
    ST_CHECK_ARG(pos, "st_positions_mask: null positions");
    ST_CHECK_ARG(!mask || aligned16(mask), "st_positions_mask: mask must be 16-byte aligned");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Rules r;
    r.k = rules->battleless_limit;
    r.cap = rules->max_plies;
    r.flags = rules->flags;
    const int blocks = (P + kRootWarps - 1) / kRootWarps;
    k_positions_mask<<<blocks, 32 * kRootWarps, kRootWarps * sizeof(RolloutSmem), s>>>(pos, P, r, mask, n_legal,
                                                                                      two_square, item_status);
    ST_CUDA(cudaGetLastError());
    return ST_OK;
}
