// Tensor-core (tcgen05) path: plan and call sequences.
#pragma once
#include <cstddef>
#include <string>
#include <vector>

#include "fgi_internal.h"

namespace fgi {

struct TcPlanInput {
    int n_batch = 0;
    const DevBatch *batches = nullptr;   // FP64-path batch table (points, actives)
    const DevAct *act = nullptr;
    const int *atom_nfn = nullptr;
    const char *tune_path = nullptr;
    bool host_only = false;              // build host tables only (no device copies)
};

struct TcPlan {
    bool built = false;
    size_t ws_bytes = 0;
    void *d_mem = nullptr;               // device tables of this path
};

int tc_build(TcPlan &t, const TcPlanInput &in, std::string *err);
void tc_free(TcPlan &t);
size_t tc_workspace_bytes(const TcPlan &t);
int tc_integrate_h(TcPlan &t, const DevPlan &P, int n_split, const double *v, double *h, void *ws,
                   cudaStream_t s, std::string *err);
int tc_density(TcPlan &t, const DevPlan &P, int n_split, const double *d, double offdiag_scale,
               double *n, void *ws, cudaStream_t s, std::string *err);

}  // namespace fgi
