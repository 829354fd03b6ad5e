// Test harness only: the env's reset sources and history on host threads
// through include/cuda_runtime.h of this directory, in the order a caller
// uses them: create (k_env_reset), history on, a setup pool (optionally
// mirrored), pinned slots (k_env_pin), reset (k_env_reset), S plies of the
// recording persistent step (k_env_run<L, true>), then the positions at
// each queried step (k_env_hist_positions).  Inputs <in>.pool ([2][M][40]),
// <in>.pins ([n][784]) and <in>.idx ([n] int32); outputs
// <out>.{action,reward,done,ply,mask,stats}, <out>.hist<t>.{pos,status},
// <out>.steps<t>.{action,done,reward} (t before now) and <out>.export (the
// snapshots of slots N-1 .. 0 now, k_env_export).
//   env_sources_on_host in out N S L wpb gpf blocks seed H M mirror n t...
#include "host_launch.h"
#include "env_dev.cu"

int main(int argc, char** argv)
{
    const std::string in = argv[1], out = argv[2];
    const int N = std::atoi(argv[3]), S = std::atoi(argv[4]), L = std::atoi(argv[5]), wpb = std::atoi(argv[6]);
    const int gpf = std::atoi(argv[7]), nblocks = std::atoi(argv[8]);
    const unsigned long long seed = std::strtoull(argv[9], nullptr, 10);
    const int H = std::atoi(argv[10]), M = std::atoi(argv[11]), mirror = std::atoi(argv[12]);
    const int npins = std::atoi(argv[13]);
    if (L != 8) { std::fprintf(stderr, "teams of 8 lanes only\n"); return 2; }
    std::vector<GameCore> core(N);
    std::vector<uint16_t> ring((size_t)N * kRing);
    std::vector<uint64_t> pi((size_t)N * kPiWords);
    std::vector<uint32_t> stats((size_t)N * 8);
    std::vector<uint32_t> hist((size_t)H * N, 0xA5A5A5A5u);
    long long d_now = 0;
    int32_t status[2] = {0, 0x7FFFFFFF};
    int32_t queue = 0;
    EnvArgs a{};
    a.core = core.data(); a.ring = ring.data(); a.pi = pi.data(); a.stats = stats.data(); a.status = status;
    a.N = N; a.k0 = (uint32_t)seed; a.k1 = (uint32_t)(seed >> 32);
    a.R.k = 100; a.R.cap = 1000; a.R.flags = kTwoSquare | kChase | kAutoreset;
    a.reset = ResetSrc{nullptr, nullptr, nullptr, 0, 0};
    a.hist = nullptr; a.now = nullptr; a.H = 0;
    launch((N + 3) / 4, 128, 4 * sizeof(SmemGame), [=] { k_env_reset(a, nullptr, nullptr, 1); });
    // history on (at step 0), pool, pins
    a.hist = hist.data(); a.H = H; a.now = &d_now;
    std::vector<uint8_t> pool;
    if (M > 0) {
        pool = load<uint8_t>(in + ".pool");
        if ((int)pool.size() != 2 * M * 40) { std::fprintf(stderr, "pool size\n"); return 2; }
        a.reset.pool = pool.data(); a.reset.pool_m = M; a.reset.pool_flags = mirror ? ST_POOL_MIRROR : 0u;
    }
    std::vector<int32_t> pin_of((size_t)N, -1);
    std::vector<RootState> recs((size_t)std::max(npins, 1));
    if (npins > 0) {
        auto raw = load<uint8_t>(in + ".pins");
        auto idx = load<int32_t>(in + ".idx");
        if ((int)raw.size() != npins * (int)sizeof(st_position) || (int)idx.size() != npins) {
            std::fprintf(stderr, "pins size\n");
            return 2;
        }
        std::vector<st_position> states((size_t)npins);
        std::memcpy(states.data(), raw.data(), raw.size());
        const EnvArgs a0 = a;
        const int32_t* ip = idx.data();
        const st_position* stp = states.data();
        RootState* rp = recs.data();
        int32_t* po = pin_of.data();
        launch((npins + 3) / 4, 128, 4 * sizeof(RolloutSmem), [=] { k_env_pin(a0, ip, npins, stp, rp, po); });
        a.reset.pin_of = pin_of.data(); a.reset.pins = recs.data();
    }
    launch((N + 3) / 4, 128, 4 * sizeof(SmemGame), [=] { k_env_reset(a, nullptr, nullptr, 0); });
    std::vector<int16_t> act((size_t)S * N), ply((size_t)S * N);
    std::vector<int8_t> rew((size_t)S * N);
    std::vector<uint8_t> done((size_t)S * N), mask((size_t)S * N * kMaskBytes);
    {
        int16_t* ap = act.data(); int8_t* rp = rew.data(); uint8_t* dp = done.data(); int16_t* pp = ply.data();
        uint8_t* mp = mask.data();
        int32_t* qp = &queue;
        // two parts per slot, the second starting mid-way through the history ring
        std::vector<int32_t> part_done((size_t)N, 0);
        int32_t* dn = part_done.data();
        const size_t sm = (size_t)wpb * 4 * kRowsRecordBytes;   // row-mode records, each followed by its mask
        launch(nblocks, 32 * wpb, sm, [=] { k_env_run<8, true>(a, qp, S, S, gpf, ap, rp, dp, pp, mp, 2, (S + 1) / 2, dn); });
    }
    d_now += S;
    dump(out + ".action", act.data(), act.size());
    dump(out + ".reward", rew.data(), rew.size());
    dump(out + ".done", done.data(), done.size());
    dump(out + ".ply", ply.data(), ply.size());
    dump(out + ".mask", mask.data(), mask.size());
    dump(out + ".stats", stats.data(), stats.size());
    for (int i = 14; i < argc; ++i) {
        const long long t = std::atoll(argv[i]);
        HistQuery q;
        q.hist = hist.data(); q.H = H; q.now = d_now; q.lo = std::max(0LL, d_now - (long long)H); q.floor = 0; q.t = t;
        std::vector<st_position> hp((size_t)N);
        std::vector<uint8_t> hs((size_t)N, 0xEE), ended((size_t)N);
        std::vector<int32_t> since((size_t)N);
        st_position* hpp = hp.data();
        uint8_t* hsp = hs.data();
        uint8_t* ep = ended.data();
        int32_t* sp = since.data();
        // teams of 4 lanes, 32 slots per block (the last block ragged when N % 32)
        std::vector<uint64_t> hpi((size_t)N * kPiWords);
        uint64_t* pp = hpi.data();
        launch((N + 31) / 32, 128, 32 * sizeof(HistSmem), [=] { k_env_hist_positions<4>(a, q, hpp, hsp, ep, sp, pp); });
        dump(out + ".hist" + std::to_string(t) + ".pos", hp.data(), hp.size());
        dump(out + ".hist" + std::to_string(t) + ".status", hs.data(), hs.size());
        if (t < d_now) {   // the record of step t
            std::vector<int16_t> ha((size_t)N);
            std::vector<uint8_t> hd((size_t)N), hm((size_t)N);
            std::vector<int8_t> hr((size_t)N);
            int16_t* hap = ha.data();
            uint8_t* hdp = hd.data();
            int8_t* hrp = hr.data();
            uint8_t* hmp = hm.data();
            launch((N + 255) / 256, 256, 0, [=] { k_env_hist_steps(N, q, hap, hdp, hrp, hmp); });
            dump(out + ".steps" + std::to_string(t) + ".action", ha.data(), ha.size());
            dump(out + ".steps" + std::to_string(t) + ".done", hd.data(), hd.size());
            dump(out + ".steps" + std::to_string(t) + ".reward", hr.data(), hr.size());
        }
    }
    {   // snapshots of every slot now
        std::vector<int32_t> idx((size_t)N);
        for (int g = 0; g < N; ++g) idx[(size_t)g] = N - 1 - g;
        std::vector<st_position> snap((size_t)N);
        const int32_t* ip = idx.data();
        st_position* sp = snap.data();
        launch((N + 3) / 4, 128, 4 * sizeof(SmemGame), [=] { k_env_export(a, ip, N, sp); });
        dump(out + ".export", snap.data(), snap.size());
    }
    std::printf("status %d %d\ndone\n", status[0], status[1]);
    return 0;
}
