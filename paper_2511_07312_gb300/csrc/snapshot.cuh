// snapshot.cuh -- device-side reading of st_position snapshots (App. B.4:
// games reset to non-initial states), shared by the env import and the
// search kernels.
#pragma once
#include "engine.cuh"
#include "stratego.h"

namespace stg {

// Warp (team of 32): read and validate snapshot `in` into G -- board, hash,
// derived bitboards, history ring and chase positions rebuilt -- writing
// this game's history ring and chase store.  Returns 0 when valid.
__device__ __forceinline__ int import_position(SmemGame* G, const st_position* in, uint16_t* ring, uint64_t* pi)
{
    const Team<32> T;
    const int lane = T.tl;
    const uint8_t* ib = reinterpret_cast<const uint8_t*>(in);
    for (int b = lane; b < 240; b += 32) reinterpret_cast<uint8_t*>(&G->c)[b] = ib[b];
    T.sync();
    int bad = 0;
    if (lane == 0) {
        GameCore& c = G->c;
        int cnt[2][12];
        for (int a = 0; a < 2; ++a)
            for (int t = 0; t < 12; ++t) cnt[a][t] = 0;
        for (int p = 0; p < 80 && !bad; ++p) {
            if (c.type[p] >= 12) { bad = 1; break; }
            cnt[p / 40][c.type[p]]++;
            if (c.sq[p] >= 100 || is_lake(c.sq[p])) bad = 2;
            if ((c.flags[p] & 1) && (c.flags[p] >> 4)) bad = 3;
        }
        const int want[12] = {1, 8, 5, 4, 4, 4, 3, 2, 1, 1, 1, 6};
        for (int a = 0; a < 2 && !bad; ++a)
            for (int t = 0; t < 12; ++t)
                if (cnt[a][t] != want[t]) bad = 4;
        c.ply = in->ply;
        c.battleless = in->battleless;
        if (!bad && (c.ply < 0 || c.battleless < 0 || c.battleless > c.ply)) bad = 6;
        c.last_battle = in->last_battle ? 1 : 0;
        c.chaser = in->chaser;
        c.chase_plies = in->chase_plies;
        if (!bad && c.chaser != kNone && c.chaser > 1) bad = 7;
        for (int p = 0; p < 2; ++p) {
            c.ts_pid[p] = in->ts_pid[p];
            c.ts_len[p] = in->ts_len[p];
            for (int k = 0; k < 4; ++k) c.ts_sq[p][k] = in->ts_sq[p][k];
            if (!bad && c.ts_pid[p] != kNone && (c.ts_pid[p] >= 80 || c.ts_len[p] < 2 || c.ts_len[p] > 4)) bad = 8;
            if (!bad && c.ts_pid[p] == kNone && c.ts_len[p] != 0) bad = 8;
            for (int k = 0; k < c.ts_len[p] && k < 4 && !bad; ++k)
                if (c.ts_sq[p][k] >= 100 || is_lake(c.ts_sq[p][k])) bad = 8;
        }
        if (!bad && c.chaser == kNone && c.chase_plies != 0) bad = 13;
        if (!bad && c.chaser != kNone && c.chase_plies < 1) bad = 9;
        c.terminated = 0;
        c.n_pi = 0;
    }
    bad = T.shfl(bad, 0);
    if (bad) return bad;
    // board, checking that no two alive pieces share a square
    for (int s = lane; s < 112; s += 32) G->board[s] = (s < 100 && is_lake(s)) ? kLake : kEmpty;
    T.sync();
    if (lane == 0) {
        for (int p = 0; p < 80 && !bad; ++p) {
            if (!(G->c.flags[p] & 1)) continue;
            if (G->board[G->c.sq[p]] != kEmpty) bad = 5;
            else G->board[G->c.sq[p]] = (uint8_t)p;
        }
    }
    bad = T.shfl(bad, 0);
    if (bad) return bad;
    const int ply = G->c.ply;
    for (int h = lane; h < kRing; h += 32)
        if (h < ply) ring[(ply - 1 - h) & (kRing - 1)] = in->hist[h];
    const uint64_t hash0 = side_hash(G, T, 0), hash1 = side_hash(G, T, 1);
    T.sync();
    if (lane == 0) {
        G->c.hash_side[0] = hash0;
        G->c.hash_side[1] = hash1;
        // chase positions: undo the chase plies from the current board,
        // recording (chaser's hash, chased side's hash) after each of the
        // chaser's plies, oldest first
        const int chaser = G->c.chaser;
        if (chaser != kNone) {
            int nt = 0;
            for (int i = 0; i < G->c.chase_plies; ++i) nt += ((ply - 1 - i) & 1) == chaser;
            if (nt > kPiCap) bad = 11;
            uint8_t b[100];
            for (int s = 0; s < 100; ++s) b[s] = G->board[s];
            uint64_t h[2] = {hash0, hash1};
            int j = 0;
            for (int i = 0; i < G->c.chase_plies && !bad; ++i) {
                const int mover = (ply - 1 - i) & 1;
                const int a = in->hist[i];
                if (a == 0xFFFF) { bad = 10; break; }
                if (mover == chaser) {
                    const int at = nt - 1 - j++;
                    pi[2 * at] = h[chaser];
                    pi[2 * at + 1] = h[1 - chaser];
                }
                const int f = a / 100, t = a % 100;
                if (f >= 100 || b[t] >= kPieces || b[f] != kEmpty || is_lake(f)) { bad = 12; break; }
                const int p = b[t];
                b[f] = (uint8_t)p;
                b[t] = kEmpty;
                h[p / 40] ^= zkey(p, t) ^ zkey(p, f);
            }
            if (!bad) G->c.n_pi = (uint8_t)nt;
        }
    }
    bad = T.shfl(bad, 0);
    T.sync();
    if (bad) return bad;
    derive_state(G, ring, pi, T);
    return 0;
}

}  // namespace stg
