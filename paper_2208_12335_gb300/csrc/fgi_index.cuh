// Device helpers that map a batch's local function indices to the stored
// values of the sparse upper-triangular matrices (CSR order by rows).
#pragma once
#include "fgi_internal.h"

namespace fgi {

// largest e in [0, n) with act[e].fn_loc <= l
__device__ __forceinline__ int find_act(const DevAct *act, int n, int l)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (act[mid].fn_loc <= l) lo = mid; else hi = mid - 1;
    }
    return lo;
}

struct FnRef {
    long long gi;   // global function
    int atom;       // global atom
    int li;         // index inside the atom
};

__device__ __forceinline__ FnRef fn_ref(const DevPlan &P, const DevAct *act, int e, int l)
{
    DevAct A = act[e];
    FnRef r;
    r.atom = A.atom;
    r.li = l - A.fn_loc;
    r.gi = P.atom_fn0[A.atom] + r.li;
    return r;
}

// Stored value of (a, b), a.gi <= b.gi.  Row a.gi holds first the rest of its
// own atom's functions (j >= i), then every neighbour atom b > a in
// ascending order; pairpos gives the start of atom b's run for the atom's
// first function.  -1 when the atom pair is not stored (its values are 0).
__device__ __forceinline__ long long value_index(const DevPlan &P, int sys, const FnRef &a,
                                                 const FnRef &b)
{
    long long rp = P.rowptr[a.gi];
    if (a.atom == b.atom) return rp + (b.gi - a.gi);
    int nat = P.sys_nat[sys];
    int pp = P.pairpos[P.sys_pair_off[sys] + (long long)P.atom_loc[a.atom] * nat + P.atom_loc[b.atom]];
    if (pp < 0) return -1;
    return rp + pp - a.li + b.li;
}

}  // namespace fgi
