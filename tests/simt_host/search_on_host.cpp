// Test harness only: runs the kernels of st_search (k_search_prep,
// k_search_offsets, k_draw_samples, k_search_rollouts on `fb` resident
// blocks, k_search_policy) on host threads through include/cuda_runtime.h
// of this directory, on P positions read from <in>.pos, and writes
// <out>.{n_moves,actions,tallies,q,pi,chosen,status}.
//   search_on_host in P S depth seed fb flags out
#include "host_launch.h"
#include "search_dev.cu"

int main(int argc, char** argv)
{
    const std::string in = argv[1], out = argv[8];
    const int P = std::atoi(argv[2]), S = std::atoi(argv[3]), depth = std::atoi(argv[4]);
    const unsigned long long seed = std::strtoull(argv[5], nullptr, 10);
    const int fb = std::atoi(argv[6]);
    const uint32_t flags = (uint32_t)std::strtoul(argv[7], nullptr, 10);
    auto raw = load<uint8_t>(in + ".pos");
    if ((int)raw.size() != P * (int)sizeof(st_position)) { std::fprintf(stderr, "input sizes\n"); return 2; }
    std::vector<st_position> pos((size_t)P);
    std::memcpy(pos.data(), raw.data(), raw.size());
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    Rules r;
    r.k = 100; r.cap = 1000; r.flags = flags;
    const double alpha = 0.002, beta = 0.02;
    std::vector<RootState> roots((size_t)P);
    std::vector<long long> offs((size_t)P + 1);
    std::vector<int32_t> n_moves((size_t)P), tallies((size_t)P * kSearchMoves * 4);
    std::vector<int16_t> actions((size_t)P * kSearchMoves), chosen((size_t)P);
    std::vector<double> q((size_t)P * kSearchMoves), pi((size_t)P * kSearchMoves);
    std::vector<uint8_t> status((size_t)P, 0xEE);
    const st_position* pp = pos.data();
    RootState* rp = roots.data();
    long long* op = offs.data();
    int32_t* np_ = n_moves.data();
    int32_t* tp = tallies.data();
    int16_t* ap = actions.data();
    int16_t* cp = chosen.data();
    double* qp = q.data();
    double* pip = pi.data();
    uint8_t* sp = status.data();
    launch((P + kRootWarps - 1) / kRootWarps, 32 * kRootWarps, kRootWarps * sizeof(RolloutSmem),
           [=] { k_search_prep(pp, P, r, rp, np_, ap, tp, qp, pip, cp, sp); });
    launch(1, kOffsetThreads, 0, [=] { k_search_offsets(np_, P, S, op); });
    std::vector<uint8_t> drawn((size_t)P * S * 40);
    uint8_t* dp = drawn.data();
    launch((unsigned)(((long long)P * S + 127) / 128), 128, 0, [=] { k_draw_samples(rp, P, S, k0, k1, nullptr, dp); });
    std::vector<uint64_t> scratch((size_t)fb * kFlatTeams * kPiWords, 0x5A5A5A5A5A5A5A5Aull);
    uint64_t* sc = scratch.data();
    launch((unsigned)fb, 32 * kFlatWarps, kFlatTeams * sizeof(FlatSmem),
           [=] { k_search_rollouts(rp, op, P, S, depth, k0, k1, nullptr, ap, r, tp, sc, dp); });
    launch((P + kPolicyWarps - 1) / kPolicyWarps, 32 * kPolicyWarps, 0,
           [=] { k_search_policy(P, S, k0, k1, nullptr, nullptr, nullptr, alpha, beta, np_, ap, tp, qp, pip, cp, sp); });
    dump(out + ".n_moves", n_moves.data(), n_moves.size());
    dump(out + ".actions", actions.data(), actions.size());
    dump(out + ".tallies", tallies.data(), tallies.size());
    dump(out + ".q", q.data(), q.size());
    dump(out + ".pi", pi.data(), pi.size());
    dump(out + ".chosen", chosen.data(), chosen.size());
    dump(out + ".status", status.data(), status.size());
    std::printf("done\n");
    return 0;
}
