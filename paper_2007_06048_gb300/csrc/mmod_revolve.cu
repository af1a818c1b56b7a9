// Binomial checkpointing schedule (Griewank 1992; Griewank & Walther 2000,
// "Algorithm 799: revolve") for reversing nsteps time steps with `snaps`
// checkpoint slots besides the initial state (which is zero and needs none).
//
// Host code only.  With S = snaps + 1 stored states in all and
// beta(S, r) = C(S + r, S) (the most steps S states can reverse when no step
// is advanced more than r times), reversing l steps from a stored state at a
// works as follows: r = the least repetition number with beta(S, r) >= l;
// advance j steps, store the state a + j in a free slot, reverse the last
// l - j steps with one slot fewer, release the slot, go back to a and reverse
// the first j steps.  The split
//     j = max(l - beta(S - 1, r), beta(S, r - 2), 1)
// keeps the last part at repetition r with S - 1 states and the first at
// repetition r - 1 with S states, which attains the minimal number of
// advanced steps r l - beta(S + 1, r - 1).  With no free slot the steps are
// reversed one by one, each from the stored state.  The schedule is kept
// iterative (an explicit task stack), so its depth is not bounded by the
// thread's stack.
#include <algorithm>
#include <vector>

#include "mmod_handle.h"

#define MMOD_API extern "C" __attribute__((visibility("default")))

namespace mmod {

namespace {

// C(S + r, S), saturated at cap + 1 (values above cap never change a
// decision).  b stays <= cap + 1 and S + k < 2^32, so b (S + k) fits.
long long binom_sat(int S, int r, long long cap) {
    if (r < 0) return 0;
    long long b = 1;
    for (int k = 1; k <= r; ++k) {
        const long long m = (long long)S + k;
        if ((double)b * (double)m / (double)k > (double)cap + 1.0) return cap + 1;
        b = b * m / k;   // C(S + k, k) = C(S + k - 1, k - 1) (S + k) / k, exact
    }
    return b;
}

struct Task {
    int kind;   // 0: reverse [a, a + l) from the state stored in `slot`; 1: release `slot`
    int a, l, slot;
};

}  // namespace

long long revolve_schedule(int nsteps, int snaps, std::vector<RevAction> *out) {
    out->clear();
    if (nsteps <= 0) return 0;
    snaps = std::max(0, std::min(snaps, nsteps - 1));
    std::vector<int> free_slots;
    for (int q = snaps - 1; q >= 0; --q) free_slots.push_back(q);
    long long advanced = 0;
    int cur = 0;   // step of the state in the working buffers (the initial state at first)
    auto restore = [&](int slot, int step) {
        if (cur != step) {
            out->push_back({MMOD_REV_RESTORE, slot, step});
            cur = step;
        }
    };
    auto advance = [&](int to) {
        if (to > cur) {
            out->push_back({MMOD_REV_ADVANCE, cur, to});
            advanced += to - cur;
            cur = to;
        }
    };
    std::vector<Task> stack{{0, 0, nsteps, -1}};
    while (!stack.empty()) {
        const Task t = stack.back();
        stack.pop_back();
        if (t.kind == 1) {
            free_slots.push_back(t.slot);
            continue;
        }
        restore(t.slot, t.a);
        if (t.l == 1) {
            out->push_back({MMOD_REV_REVERSE, t.a, 0});
            continue;
        }
        if (free_slots.empty()) {
            for (int i = t.l - 1; i >= 0; --i) {
                restore(t.slot, t.a);
                advance(t.a + i);
                out->push_back({MMOD_REV_REVERSE, t.a + i, 0});
            }
            continue;
        }
        const int S = (int)free_slots.size() + 1;
        const long long cap = t.l;
        int r = 0;
        while (binom_sat(S, r, cap) < t.l) ++r;
        long long j = std::max<long long>(t.l - binom_sat(S - 1, r, cap), 1);
        if (r >= 2) j = std::max<long long>(j, binom_sat(S, r - 2, cap));
        j = std::min<long long>(j, t.l - 1);
        advance(t.a + (int)j);
        const int q = free_slots.back();
        free_slots.pop_back();
        out->push_back({MMOD_REV_SAVE, q, t.a + (int)j});
        // executed in reverse order of pushing: the last part, the release of
        // q, then the first part from the caller's state
        stack.push_back({0, t.a, (int)j, t.slot});
        stack.push_back({1, 0, 0, q});
        stack.push_back({0, t.a + (int)j, t.l - (int)j, q});
    }
    return advanced;
}

}  // namespace mmod

MMOD_API mmod_status mmod_revolve_schedule(int nsteps, int snaps, int *actions, long long cap, long long *count,
                                           long long *advanced) {
    if (nsteps < 0 || snaps < 0 || cap < 0 || (cap > 0 && !actions)) return MMOD_ERR_ARG;
    std::vector<mmod::RevAction> sched;
    const long long adv = mmod::revolve_schedule(nsteps, snaps, &sched);
    if (count) *count = (long long)sched.size();
    if (advanced) *advanced = adv;
    if ((long long)sched.size() > cap) return actions ? MMOD_ERR_ARG : MMOD_OK;
    for (size_t q = 0; q < sched.size(); ++q) {
        actions[3 * q] = sched[q].kind;
        actions[3 * q + 1] = sched[q].a;
        actions[3 * q + 2] = sched[q].b;
    }
    return MMOD_OK;
}
