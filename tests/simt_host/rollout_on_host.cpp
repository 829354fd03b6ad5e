// Test harness only: runs the rollout kernels of st_rollout (k_roots, the
// draw-ahead k_draw_samples when asked, k_rollout_flat on a grid of `fb`
// resident blocks striding over the units) on host threads through
// include/cuda_runtime.h of this directory, on P positions read from
// <in>.pos, and writes <out>.{tallies,status}; then st_belief_sample's
// k_belief (a block per position, __syncthreads) into <out>.types and
// st_positions_mask's k_positions_mask into <out>.{mask,n_legal,two_square}.
//   rollout_on_host in P K depth seed draw_ahead fb flags out
#include "host_launch.h"
#include "search_dev.cu"

int main(int argc, char** argv)
{
    const std::string in = argv[1], out = argv[9];
    const int P = std::atoi(argv[2]), K = std::atoi(argv[3]), depth = std::atoi(argv[4]);
    const unsigned long long seed = std::strtoull(argv[5], nullptr, 10);
    const int draw_ahead = std::atoi(argv[6]), fb = std::atoi(argv[7]);
    const uint32_t flags = (uint32_t)std::strtoul(argv[8], nullptr, 10);
    auto raw = load<uint8_t>(in + ".pos");
    if ((int)raw.size() != P * (int)sizeof(st_position)) { std::fprintf(stderr, "input sizes\n"); return 2; }
    std::vector<st_position> pos((size_t)P);
    std::memcpy(pos.data(), raw.data(), raw.size());
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    Rules r;
    r.k = 100; r.cap = 1000; r.flags = flags;
    std::vector<RootState> roots((size_t)P);
    std::vector<uint8_t> status((size_t)P, 0xEE);
    std::vector<int32_t> tallies((size_t)P * 4, 0);
    const st_position* pp = pos.data();
    RootState* rp = roots.data();
    uint8_t* sp = status.data();
    launch((P + kRootWarps - 1) / kRootWarps, 32 * kRootWarps, kRootWarps * sizeof(RolloutSmem),
           [=] { k_roots(pp, P, rp, sp); });
    const long long units = (long long)P * K;
    std::vector<uint8_t> drawn;
    const uint8_t* ty = nullptr;
    if (draw_ahead) {
        drawn.assign((size_t)units * 40, 0);
        uint8_t* dp = drawn.data();
        launch((unsigned)((units + 127) / 128), 128, 0, [=] { k_draw_samples(rp, P, K, k0, k1, nullptr, dp); });
        ty = drawn.data();
    }
    std::vector<uint64_t> scratch((size_t)fb * kFlatTeams * kPiWords, 0x5A5A5A5A5A5A5A5Aull);
    uint64_t* sc = scratch.data();
    int32_t* tp = tallies.data();
    launch((unsigned)fb, 32 * kFlatWarps, kFlatTeams * sizeof(FlatSmem),
           [=] { k_rollout_flat(rp, P, K, depth, k0, k1, nullptr, ty, r, tp, sc); });
    dump(out + ".tallies", tallies.data(), tallies.size());
    dump(out + ".status", status.data(), status.size());
    std::vector<uint8_t> types((size_t)P * K * 40, 0xEE), bstatus((size_t)P, 0xEE);
    uint8_t* tp2 = types.data();
    uint8_t* bs = bstatus.data();
    launch((unsigned)P, 128, 0, [=] { k_belief(pp, P, K, k0, k1, nullptr, tp2, bs); });
    dump(out + ".types", types.data(), types.size());
    std::vector<uint8_t> mask((size_t)P * kMaskBytes, 0xEE), two((size_t)P, 0xEE), mstatus((size_t)P, 0xEE);
    std::vector<int32_t> n_legal((size_t)P, -7);
    uint8_t* mp = mask.data();
    uint8_t* twp = two.data();
    uint8_t* msp = mstatus.data();
    int32_t* nlp = n_legal.data();
    launch((P + kRootWarps - 1) / kRootWarps, 32 * kRootWarps, kRootWarps * sizeof(RolloutSmem),
           [=] { k_positions_mask(pp, P, r, mp, nlp, twp, msp); });
    dump(out + ".mask", mask.data(), mask.size());
    dump(out + ".n_legal", n_legal.data(), n_legal.size());
    dump(out + ".two_square", two.data(), two.size());
    std::printf("done\n");
    return 0;
}
