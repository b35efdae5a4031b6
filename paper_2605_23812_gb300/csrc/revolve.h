// revolve.h -- binomial checkpointing schedule for the reverse sweep of the discrete adjoint
// (Sec. 3.2: the adjoint runs backward in time over the stored forward trajectory; checkpointing
// trades recomputation for memory).  Host-only C++, no CUDA.
//
// State k is the forward state after k time steps.  Reversing step k (k -> k+1) needs state k.
// Slot 0 always holds state 0; slots 1 .. S-1 are free.  With s snapshots (the one holding the
// segment's first state included) and repetition number r, at most beta(s, r) = C(s + r, s) steps
// can be reversed with every step advanced at most r times (Griewank's bound).  The recursion
// rev(a, b, c) with c free slots, i.e. s = c + 1:
//   b - a == 1 : restore state a, reverse step a
//   c == 0     : for k = b-1 .. a: restore a, advance to k, reverse step k
//   otherwise  : advance a -> m = a + k, store m in slot S-c, rev(m, b, c-1), then rev(a, m, c).
// Cost (forward steps) of a segment of n steps: T(n, c) = sum_{m=2..n} rep(c+1, m), rep(s, m) the
// least r with beta(s, r) >= m; it is reached by the split
//   k = max(beta(s, r-2), n - beta(s-1, r), 1),  r = rep(s, n).
// The first descent along the right spine is the initial forward sweep, whose advances are paid
// anyway; its splits minimise Tspine(n-k, c-1) + T(k, c) with Tspine(n, c) = T(n+1, c) - n.
// Both rules were checked against exhaustive minimisation over every split for small n and c.
#pragma once

#include <algorithm>
#include <cstdint>
#include <vector>

namespace envar {

// C(s + r, s), saturated at `cap`; 0 for r < 0
inline long long revolve_beta(int s, int r, long long cap)
{
    if (r < 0) return 0;
    double b = 1.0;
    for (int i = 1; i <= s; ++i) {
        b = b * (double)(r + i) / (double)i;
        if (b > (double)cap) return cap;
    }
    return (long long)(b + 0.5);
}

// least r with beta(s, r) >= m
inline int revolve_rep(int s, long long m)
{
    int r = 0;
    while (revolve_beta(s, r, m) < m) ++r;
    return r;
}

// T(n, c): forward steps to reverse n steps from a restored state with c free slots
inline long long revolve_cost(long long n, int c)
{
    const int s = c + 1;
    long long t = 0, lo = 1;   // m in (beta(s, r-1), beta(s, r)] has rep(s, m) = r
    for (int r = 1; lo < n; ++r) {
        const long long hi = std::min(revolve_beta(s, r, n), n);
        t += (long long)r * (hi - lo);
        lo = hi;
    }
    return t;
}

// Steps to advance from a before placing the next checkpoint, for n = b - a > 1 and c > 0 free
// slots; `spine`: the advances are part of the initial sweep.
inline long long revolve_split(long long n, int c, bool spine)
{
    if (c >= n - 1) return 1;   // a slot for every state: no recomputation
    const int s = c + 1;
    if (!spine) {
        const int r = revolve_rep(s, n);
        long long k = std::max(revolve_beta(s, r - 2, n), n - revolve_beta(s - 1, r, n));
        return std::max(1LL, std::min(k, n - 1));
    }
    long long best_k = 1, best = -1;
    for (long long k = 1; k < n; ++k) {
        const long long v = (revolve_cost(n - k + 1, c - 1) - (n - k)) + revolve_cost(k, c);
        if (best < 0 || v < best) { best = v; best_k = k; }
    }
    return best_k;
}

// Executor interface: advance(from, to) runs the forward from the working state `from` to `to`;
// store(slot, k) copies the working state k into a slot; restore(slot, k) copies it back;
// reverse(k) reverses step k with the working state k.  Each returns 0 or an error code.
template <class Ex>
int revolve_rev(Ex &ex, long long a, long long b, int c, int slot_a, int S, bool spine)
{
    const long long n = b - a;
    int rc;
    if (n <= 0) return 0;
    if (n == 1) {
        if ((rc = ex.restore(slot_a, a))) return rc;
        return ex.reverse(a);
    }
    if (c == 0) {
        for (long long k = b - 1; k >= a; --k) {
            if ((rc = ex.restore(slot_a, a))) return rc;
            if (k > a && (rc = ex.advance(a, k))) return rc;
            if ((rc = ex.reverse(k))) return rc;
        }
        return 0;
    }
    const long long m = a + revolve_split(n, c, spine);
    const int slot_m = S - c;
    if (!spine) {
        if ((rc = ex.restore(slot_a, a))) return rc;
        if ((rc = ex.advance(a, m))) return rc;
        if ((rc = ex.store(slot_m, m))) return rc;
    }
    if ((rc = revolve_rev(ex, m, b, c - 1, slot_m, S, spine))) return rc;
    return revolve_rev(ex, a, m, c, slot_a, S, false);
}

// Checkpoint positions of the right spine (the initial forward sweep), in increasing order;
// spine_slot[i] is the slot of spine_pos[i].
inline void revolve_spine(long long n, int S, std::vector<long long> *pos, std::vector<int> *slot)
{
    pos->clear();
    slot->clear();
    long long a = 0;
    int c = S - 1;
    while (n - a > 1 && c > 0) {
        a += revolve_split(n - a, c, true);
        pos->push_back(a);
        slot->push_back(S - c);
        --c;
    }
}

// Dry run: checks the schedule (every step reversed once, in order n-1 .. 0, always from the
// right state; slots in range) and counts forward steps, stores and restores.
struct RevolveCheck {
    long long n = 0;
    int S = 0;
    long long cur = 0;           // state in the working buffers (-1: none)
    long long next_rev = 0;      // step expected next
    long long fwd = 0, stores = 0, restores = 0, max_slot = 0;
    std::vector<long long> slot_state;
    bool ok = true;
    int advance(long long from, long long to)
    {
        if (cur != from || to <= from) ok = false;
        fwd += to - from;
        cur = to;
        return 0;
    }
    int store(int slot, long long k)
    {
        if (slot < 1 || slot >= S || cur != k) ok = false;
        else slot_state[slot] = k;
        max_slot = std::max<long long>(max_slot, slot);
        ++stores;
        return 0;
    }
    int restore(int slot, long long k)
    {
        if (slot < 0 || slot >= S || slot_state[slot] != k) ok = false;
        ++restores;
        cur = k;
        return 0;
    }
    int reverse(long long k)
    {
        if (cur != k || k != next_rev) ok = false;
        --next_rev;
        cur = -1;
        return 0;
    }
};

// Runs the whole schedule against RevolveCheck.  Returns forward steps beyond the initial sweep
// (recomputation), or -1 if the schedule is wrong.
inline long long revolve_dry_run(long long n, int S, long long *stores, long long *restores)
{
    RevolveCheck ck;
    ck.n = n;
    ck.S = S;
    ck.slot_state.assign((size_t)S, -1);
    ck.slot_state[0] = 0;
    std::vector<long long> pos;
    std::vector<int> slot;
    revolve_spine(n, S, &pos, &slot);
    long long prev = 0;
    for (size_t i = 0; i < pos.size(); ++i) {   // initial sweep 0 -> n, storing the spine
        if (slot[i] < 1 || slot[i] >= S || pos[i] <= prev || pos[i] >= n) ck.ok = false;
        else ck.slot_state[(size_t)slot[i]] = pos[i];
        prev = pos[i];
    }
    ck.cur = n;
    ck.next_rev = n - 1;
    revolve_rev(ck, 0, n, S - 1, 0, S, true);
    if (ck.next_rev != -1) ck.ok = false;
    if (stores) *stores = ck.stores + (long long)pos.size();
    if (restores) *restores = ck.restores;
    return ck.ok ? ck.fwd : -1;
}

} // namespace envar
