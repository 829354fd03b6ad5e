// Test harness only: one serving batch on host threads through
// include/cuda_runtime.h of this directory: k_serve_roots, then
// k_serve_rollouts on `fb` resident blocks striding over the batch's units,
// the last unit of each request publishing its tallies and completion word.
// Requests from <in>.pos ([R][784]) and <in>.req ([R] x {K, depth, seed lo,
// seed hi, stream id} int32); writes <out>.{tallies,done}.
//   serve_on_host in R fb out
#include "host_launch.h"
#include "serve_dev.cu"

int main(int argc, char** argv)
{
    const std::string in = argv[1], out = argv[4];
    const int R = std::atoi(argv[2]), fb = std::atoi(argv[3]);
    auto raw = load<uint8_t>(in + ".pos");
    auto req = load<int32_t>(in + ".req");
    if ((int)raw.size() != R * (int)sizeof(st_position) || (int)req.size() != 5 * R) {
        std::fprintf(stderr, "input sizes\n");
        return 2;
    }
    std::vector<Staged> staged((size_t)R);
    std::vector<BatchEntry> entries((size_t)R);
    long long units = 0;
    int sample_base = 0;
    for (int i = 0; i < R; ++i) {
        std::memcpy(&staged[(size_t)i].pos, raw.data() + (size_t)i * sizeof(st_position), sizeof(st_position));
        ReqDesc& d = staged[(size_t)i].desc;
        std::memset(&d, 0, sizeof(d));
        d.K = req[5 * i]; d.depth = req[5 * i + 1];
        d.k0 = (uint32_t)req[5 * i + 2]; d.k1 = (uint32_t)req[5 * i + 3]; d.stream = (uint32_t)req[5 * i + 4];
        d.seq = 1000u + (uint32_t)i;
        d.sample_base = sample_base;
        d.remaining = d.K;
        entries[(size_t)i].slot = i;
        entries[(size_t)i].unit_begin = (int32_t)units;
        units += d.K;
        sample_base += d.K;
    }
    Rules rl;
    rl.k = 100; rl.cap = 1000; rl.flags = kTwoSquare | kChase;
    std::vector<RootState> roots((size_t)R);
    std::vector<ReqDesc> descs((size_t)R);
    std::vector<SampleRec> samples((size_t)std::max(sample_base, 1));
    std::vector<int32_t> host_tallies((size_t)R * 4, 0x7EEEEEEE);
    std::vector<uint32_t> host_done((size_t)R, 0);
    std::vector<uint64_t> scratch((size_t)fb * kServeTeams * kPiWords, 0x5A5A5A5A5A5A5A5Aull);
    const BatchEntry* ep = entries.data();
    const Staged* sp = staged.data();
    RootState* rp = roots.data();
    ReqDesc* dp = descs.data();
    SampleRec* smp = samples.data();
    int32_t* ht = host_tallies.data();
    uint32_t* hd = host_done.data();
    uint64_t* sc = scratch.data();
    launch((R + 3) / 4, 128, 4 * sizeof(RolloutSmem), [=] { k_serve_roots(ep, R, sp, rp, dp, ht, hd); });
    if (units > 0)
        launch((unsigned)fb, 32 * kServeWarps, kServeTeams * sizeof(FlatSmem),
               [=] { k_serve_rollouts(ep, R, units, rp, dp, smp, rl, ht, hd, sc); });
    dump(out + ".tallies", host_tallies.data(), host_tallies.size());
    dump(out + ".done", host_done.data(), host_done.size());
    std::printf("done\n");
    return 0;
}
