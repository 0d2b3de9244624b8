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
    long long rp;   // index of the first stored value of row gi
    int atom;       // global atom
    int li;         // index inside the atom
    int loc;        // atom index inside its system
    int pad;
};

__device__ __forceinline__ FnRef fn_ref(const DevPlan &P, const DevAct *act, int e, int l)
{
    DevAct A = act[e];
    FnRef r;
    r.atom = A.atom;
    r.li = l - A.fn_loc;
    r.gi = P.atom_fn0[A.atom] + r.li;
    r.rp = P.rowptr[r.gi];
    r.loc = P.atom_loc[A.atom];
    r.pad = 0;
    return r;
}

// value_index with the system's pair table and atom count already looked up
__device__ __forceinline__ long long value_index_pp(const int *pairpos_sys, int nat, const FnRef &a, const FnRef &b)
{
    if (a.atom == b.atom) return a.rp + (b.gi - a.gi);
    const int pp = __ldg(pairpos_sys + (long long)a.loc * nat + b.loc);
    if (pp < 0) return -1;
    return a.rp + pp - a.li + b.li;
}

// Stored value of (a, b), a.gi <= b.gi.  Row a.gi holds first the rest of its
// own atom's functions (j >= i), then every neighbour atom b > a in
// ascending order; pairpos gives the start of atom b's run for the atom's
// first function.  -1 when the atom pair is not stored (its values are 0).
__device__ __forceinline__ long long value_index(const DevPlan &P, int sys, const FnRef &a,
                                                 const FnRef &b)
{
    return value_index_pp(P.pairpos + P.sys_pair_off[sys], P.sys_nat[sys], a, b);
}

}  // namespace fgi
