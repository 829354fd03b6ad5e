// search.cu -- belief samples of the opponent's hidden pieces and random
// rollouts from each sample (App. E "Search", steps 1-2, with the uniform
// posterior over consistent assignments in place of the belief network and a
// uniform random policy in place of the move network).
//
// k_belief: one block per position; the position is read once into shared
// memory, its hidden-piece plan is built once, and every thread then draws
// whole samples (Fisher-Yates over at most 40 pieces) from its own Philox
// stream.
// st_rollout: k_roots imports every position once (one warp each) into a
// root record in HBM; k_rollout_flat runs one 8-lane team per (position,
// sample), copying the root into shared memory, so a single position's
// samples spread over the whole GPU.  A rollout keeps no history ring (its
// last two moves start from the root's).
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
constexpr int kFlatLanes = 8;                              // one rollout per 8-lane team
constexpr int kFlatWarps = 2;
constexpr int kFlatTeams = 32 * kFlatWarps / kFlatLanes;   // rollouts per block

__global__ void k_roots(const st_position* pos, int P, RootState* roots, uint8_t* status)
{
    extern __shared__ __align__(16) unsigned char smem[];
    RolloutSmem* S = reinterpret_cast<RolloutSmem*>(smem) + (threadIdx.x >> 5);
    const int p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (p >= P) return;
    build_root(S, pos + p, roots + p);
    if (lane_id() == 0 && status) status[p] = roots[p].bad ? 1 : 0;
}

// One (position, sample) unit per 8-lane team; consecutive teams of a block
// share a position, so its root and plan come mostly from L1.  A rollout
// keeps no history ring (its last two moves start from the root's).
__global__ void k_rollout_flat(const RootState* roots, int P, int K, int depth, uint32_t k0, uint32_t k1,
                               const uint32_t* stream_ids, const uint8_t* types_in, Rules Rl, int32_t* tallies)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const Team<kFlatLanes> T;
    FlatSmem* S = reinterpret_cast<FlatSmem*>(smem) + threadIdx.x / kFlatLanes;
    const long long u = (long long)blockIdx.x * kFlatTeams + threadIdx.x / kFlatLanes;
    if (u >= (long long)P * K) return;
    const int p = (int)(u / K), k = (int)(u - (long long)p * K);
    const RootState* R = roots + p;
    if (R->bad) return;
    const uint32_t stream = stream_ids ? stream_ids[p] : (uint32_t)p;
    const uint8_t* t = types_in ? types_in + ((size_t)p * K + k) * 40 : nullptr;
    const int out = rollout_one(&S->g, S->types, S->pi, (uint16_t*)nullptr, T, R, &R->plan, t, depth, k0, k1, stream,
                                (uint32_t)k, Rl);
    if (T.leader()) atomicAdd(&tallies[4 * (size_t)p + out], 1);
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
    if (err == cudaSuccess && K > 0) {
        const long long units = (long long)P * K;
        const long long fb = (units + kFlatTeams - 1) / kFlatTeams;
        k_rollout_flat<<<(unsigned)fb, 32 * kFlatWarps, kFlatTeams * sizeof(FlatSmem), s>>>(
            roots, P, K, depth, (uint32_t)seed, (uint32_t)(seed >> 32), stream_ids, types, r, tallies);
        err = cudaGetLastError();
    }
    cudaFreeAsync(roots, s);
    if (err != cudaSuccess) {
        stg::set_error("st_rollout: launch failed: %s", cudaGetErrorString(err));
        return ST_ERR_CUDA;
    }
    return ST_OK;
}
