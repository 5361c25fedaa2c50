// Parallel block-pivot orderings of the two-level algorithms (Sec. 4), built
// from their definitions.
//
// Pair sets. With nbl = 2p blocks numbered 1..nbl, every parallel step is a
// perfect matching of the blocks:
//   * modulus (Sec. 4.1): step t pairs the blocks whose indices sum to
//     t + 1 modulo nbl; when that residue is even, two blocks are their own
//     partners (2i = t + 1 mod nbl), they lie p apart, and the process that
//     would idle transforms that pair of the p-th block superdiagonal (the
//     pairs visited twice per sweep). nbl steps per sweep.
//   * round robin (Sec. 4.2): the tournament schedule with block nbl fixed:
//     step t pairs the blocks 1..nbl-1 whose indices sum to t + 2 modulo
//     nbl - 1, and the block that is its own partner meets block nbl. nbl - 1
//     steps per sweep.
// Both sets are the same in every sweep; the first step of either is the
// main block antidiagonal (i + j = nbl + 1).
//
// Processes. Process q starts the first sweep on blocks (q + 1, nbl - q)
// (Sec. 4). Between steps the processes form a ring: each keeps one block and
// receives the other from one neighbour, the neighbour above (q + 1) in odd
// sweeps and below (q - 1) in even ones, so the pair of process q in the next
// step is the one that meets both its current pair and that neighbour's. With
// two processes each is the other's neighbour on both sides and the ring does
// not decide; process 0 then keeps the lower-numbered of its blocks.
//
// On one GPU the ring shift becomes a relabelling: the table records, per
// step, the pair each process holds, and every pair of a step runs in the same
// launch.
#include <stdint.h>

#include <vector>

namespace jj {

namespace {

// partner[b] (1-based) of every block in step t of the ordering.
void step_partners(int nbl, int order, int t, std::vector<int> &partner) {
    partner.assign(nbl + 1, 0);
    if (order == 1) {
        const int r = (t + 1) % nbl;
        std::vector<int> self;
        for (int i = 1; i <= nbl; ++i) {
            int j = ((r - i) % nbl + nbl) % nbl;  // i + j = r (mod nbl), j in 1..nbl
            if (j == 0) j = nbl;
            if (j == i)
                self.push_back(i);
            else
                partner[i] = j;
        }
        if (self.size() == 2) {  // even residue: the pair of the p-th superdiagonal
            partner[self[0]] = self[1];
            partner[self[1]] = self[0];
        }
    } else {
        const int M = nbl - 1;
        const int r = (t + 2) % M;
        for (int i = 1; i <= M; ++i) {
            int j = ((r - i) % M + M) % M;
            if (j == 0) j = M;
            if (j == i) {
                partner[i] = nbl;
                partner[nbl] = i;
            } else {
                partner[i] = j;
            }
        }
    }
}

}  // namespace

// Pairs (0-based, i < j) of sweep `sweep` (>= 1): steps x (nbl/2) x 2 ints,
// pair q of a step being the pivot of process q. Returns the number of steps,
// or -1 for invalid arguments.
int schedule_pairs(int nbl, int order, int sweep, int32_t *pairs) {
    if (nbl < 2 || (nbl & 1) || sweep < 1 || (order != 0 && order != 1)) return -1;
    const int p = nbl / 2;
    const int steps = order == 1 ? nbl : nbl - 1;
    std::vector<int> a(p), b(p), na(p), nb(p), partner;
    for (int q = 0; q < p; ++q) {
        a[q] = q + 1;
        b[q] = nbl - q;
    }
    for (int sw = 1; sw <= sweep; ++sw) {
        const int dir = (sw & 1) ? 1 : p - 1;  // neighbour that sends: q + 1 (odd), q - 1 (even)
        for (int t = 0; t < steps; ++t) {
            if (sw == sweep && pairs) {
                for (int q = 0; q < p; ++q) {
                    pairs[2 * (t * p + q)] = (a[q] < b[q] ? a[q] : b[q]) - 1;
                    pairs[2 * (t * p + q) + 1] = (a[q] < b[q] ? b[q] : a[q]) - 1;
                }
                if (t == steps - 1) break;
            }
            step_partners(nbl, order, t + 1 < steps ? t + 1 : 0, partner);
            if (p == 1) continue;
            if (p == 2) {
                const int keep = a[0] < b[0] ? a[0] : b[0];
                na[0] = keep;
                nb[0] = partner[keep];
                const int other = (partner[keep] == a[1]) ? b[1] : a[1];
                na[1] = other;
                nb[1] = partner[other];
            } else {
                for (int q = 0; q < p; ++q) {
                    const int s = (q + dir) % p;
                    // the block of q whose next partner the neighbour holds now
                    const bool ka = partner[a[q]] == a[s] || partner[a[q]] == b[s];
                    const bool kb = partner[b[q]] == a[s] || partner[b[q]] == b[s];
                    if (ka == kb) return -1;  // not a ring shift (never for these orderings)
                    const int keep = ka ? a[q] : b[q];
                    na[q] = keep;
                    nb[q] = partner[keep];
                }
            }
            a.swap(na);
            b.swap(nb);
        }
    }
    return steps;
}

}  // namespace jj

extern "C" int32_t jjacobi_schedule(int32_t nbl, int32_t order, int32_t sweep, int32_t *pairs) {
    return jj::schedule_pairs(nbl, order, sweep, pairs);
}
