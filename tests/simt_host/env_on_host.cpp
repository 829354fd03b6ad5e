// Test harness only: runs the env's reset kernel and its persistent step
// kernel (k_env_run) on host threads through include/cuda_runtime.h of this
// directory.  N slots, S plies in one launch of `blocks` blocks of `wpb`
// warps with teams of L lanes, every ply's outputs kept (ring of S rows) and
// written to <out>.{action,reward,done,ply,mask,stats} for comparison with
// the oracle.
//   env_on_host N S L wpb gpf blocks seed out [actions]
// NSPLIT in the environment (default 1) sets the persistent launch's parts
// per slot.
// With an actions file ([S][N] int16, -1 = the random policy) the plain
// path runs instead: one k_env_step launch per ply (teams of 4 lanes, 4
// warps per block) with those actions supplied.
#include "host_launch.h"
#include "env_dev.cu"

template <int L>
static void run(EnvArgs a, int32_t* queue, int S, int gpf, int wpb, int blocks, int16_t* act, int8_t* rew, uint8_t* done,
                int16_t* ply, uint8_t* mask, int nsplit, int32_t* part_done)
{
    const size_t sm = (size_t)wpb * (32 / L) * kRowsRecordBytes;   // row-mode records, each followed by its mask
    launch(blocks, 32 * wpb, sm,
           [=] { k_env_run<L, false>(a, queue, S, S, gpf, act, rew, done, ply, mask, nsplit, (S + nsplit - 1) / nsplit, part_done); });
}

int main(int argc, char** argv)
{
    const int N = std::atoi(argv[1]), S = std::atoi(argv[2]), L = std::atoi(argv[3]), wpb = std::atoi(argv[4]);
    const int gpf = std::atoi(argv[5]), blocks = std::atoi(argv[6]);
    const unsigned long long seed = std::strtoull(argv[7], nullptr, 10);
    const std::string out = argv[8];
    std::vector<GameCore> core(N);
    std::vector<uint16_t> ring((size_t)N * kRing);
    std::vector<uint64_t> pi((size_t)N * kPiWords);
    std::vector<uint32_t> stats((size_t)N * 8);
    int32_t status[2] = {0, 0x7FFFFFFF};
    // QUEUE0: the persistent launch's first work unit (N with NSPLIT 2 runs
    // only second parts, whose first parts never finish: every wait runs out)
    int32_t queue = std::getenv("QUEUE0") ? std::atoi(std::getenv("QUEUE0")) : 0;
    const int nsplit = std::getenv("NSPLIT") ? std::atoi(std::getenv("NSPLIT")) : 1;
    std::vector<int32_t> part_done((size_t)N, 0);
    EnvArgs a{};
    a.core = core.data(); a.ring = ring.data(); a.pi = pi.data(); a.stats = stats.data(); a.status = status;
    a.N = N; a.k0 = (uint32_t)seed; a.k1 = (uint32_t)(seed >> 32);
    a.R.k = 100; a.R.cap = 1000; a.R.flags = kTwoSquare | kChase | kAutoreset;
    a.reset = ResetSrc{nullptr, nullptr, nullptr, 0, 0};
    a.hist = nullptr; a.now = nullptr; a.H = 0;
    // creation: every slot reset (teams of 32, 4 per block)
    launch((N + 3) / 4, 128, 4 * sizeof(SmemGame), [=] { k_env_reset(a, nullptr, nullptr, 1); });
    std::vector<int16_t> act((size_t)S * N), ply((size_t)S * N);
    std::vector<int8_t> rew((size_t)S * N);
    std::vector<uint8_t> done((size_t)S * N), mask((size_t)S * N * kMaskBytes);
    if (argc > 9) {
        const std::vector<int16_t> given = load<int16_t>(argv[9]);
        if ((long long)given.size() != (long long)S * N) { std::fprintf(stderr, "actions size\n"); return 2; }
        for (int j = 0; j < S; ++j) {
            const size_t o = (size_t)j * N;
            const int16_t* gv = given.data() + o;
            int16_t* ao = act.data() + o;
            int8_t* ro = rew.data() + o;
            uint8_t* dn = done.data() + o;
            int16_t* po = ply.data() + o;
            uint8_t* mo = mask.data() + o * kMaskBytes;
            launch((N + 31) / 32, 128, 32 * sizeof(SmemGame), [=] { k_env_step<4>(a, gv, ao, ro, dn, po, mo); });
        }
    } else if (L == 8) run<8>(a, &queue, S, gpf, wpb, blocks, act.data(), rew.data(), done.data(), ply.data(), mask.data(), nsplit,
                       part_done.data());
    else if (L == 4) run<4>(a, &queue, S, gpf, wpb, blocks, act.data(), rew.data(), done.data(), ply.data(), mask.data(), nsplit,
                       part_done.data());
    else if (L == 16) run<16>(a, &queue, S, gpf, wpb, blocks, act.data(), rew.data(), done.data(), ply.data(), mask.data(), nsplit,
                       part_done.data());
    else run<32>(a, &queue, S, gpf, wpb, blocks, act.data(), rew.data(), done.data(), ply.data(), mask.data(), nsplit,
                 part_done.data());
    dump(out + ".action", act.data(), act.size());
    dump(out + ".reward", rew.data(), rew.size());
    dump(out + ".done", done.data(), done.size());
    dump(out + ".ply", ply.data(), ply.size());
    dump(out + ".mask", mask.data(), mask.size());
    dump(out + ".stats", stats.data(), stats.size());
    std::printf("status %d %d\n", status[0], status[1]);
    return 0;
}
