// Parallel block-pivot orderings of the two-level algorithms (Sec. 4):
// Initialize (Alg. 4.1), the modified modulus step MMStep (Alg. 4.2) and the
// modified round-robin step RLStep (Alg. 4.3), run for every process of a
// ring of p = nbl/2 processes. On one GPU the ring shift that follows each
// step becomes a relabelling: the table records, per step, the block pair
// each process holds, and every pair of a step runs in the same launch.
#include <stdint.h>

#include <vector>

namespace jj {

namespace {

struct PivotState {
    int ip, jp, i_blk, j_blk;
};

// Alg. 4.1: process `rank` starts the sweep on blocks (rank+1, nbl-rank).
PivotState initialize(int rank, int nbl) {
    PivotState s;
    s.ip = rank + 1;
    s.i_blk = s.ip;
    s.jp = nbl - rank;
    s.j_blk = s.jp;
    return s;
}

// Alg. 4.2: next pivot of the modified modulus strategy.
void mm_step(int nbl, PivotState &s) {
    if (s.ip + s.jp > nbl) {
        s.ip += 1;
        if (s.ip == s.jp) {
            s.ip -= nbl / 2;
            s.jp = s.ip;
        }
        s.i_blk = s.ip;
    } else {
        s.jp += 1;
        s.j_blk = s.jp;
    }
}

// Alg. 4.3: next pivot of the modified round-robin strategy (the swap flag
// only renumbers the pair so that i_blk < j_blk, which the table does anyway).
void rl_step(int nbl, PivotState &s) {
    if (s.ip + s.jp > nbl) {
        if (s.jp < nbl) {
            s.ip += 1;
            if (s.ip < s.jp) {
                s.i_blk = s.ip;
            } else {
                s.ip = s.jp;
                s.i_blk = s.j_blk;
                s.jp = nbl;
                s.j_blk = s.jp;
            }
        } else if (s.ip > nbl / 2) {
            s.ip = s.ip - nbl / 2 + 1;
            s.i_blk = s.ip;
        } else {
            s.jp = s.ip + 1;
            s.j_blk = s.jp;
        }
    } else {
        s.jp += 1;
        s.j_blk = s.jp;
    }
}

}  // namespace

// Pairs (0-based, i < j) of sweep `sweep` (>= 1): steps x (nbl/2) x 2 ints.
// Returns the number of steps, or -1 for invalid arguments.
int schedule_pairs(int nbl, int order, int sweep, int32_t *pairs) {
    if (nbl < 2 || (nbl & 1) || sweep < 1 || (order != 0 && order != 1)) return -1;
    const int p = nbl / 2;
    const int steps = order == 1 ? nbl : nbl - 1;
    std::vector<PivotState> st(p);
    for (int q = 0; q < p; ++q) st[q] = initialize(q, nbl);
    for (int sw = 1; sw <= sweep; ++sw) {
        for (int t = 0; t < steps; ++t) {
            if (sw == sweep && pairs) {
                for (int q = 0; q < p; ++q) {
                    int a = st[q].i_blk - 1, b = st[q].j_blk - 1;
                    if (a > b) {
                        const int x = a;
                        a = b;
                        b = x;
                    }
                    pairs[2 * (t * p + q)] = a;
                    pairs[2 * (t * p + q) + 1] = b;
                }
            }
            for (int q = 0; q < p; ++q) {
                if (order == 1)
                    mm_step(nbl, st[q]);
                else
                    rl_step(nbl, st[q]);
            }
        }
    }
    return steps;
}

}  // namespace jj

extern "C" int32_t jjacobi_schedule(int32_t nbl, int32_t order, int32_t sweep, int32_t *pairs) {
    return jj::schedule_pairs(nbl, order, sweep, pairs);
}
