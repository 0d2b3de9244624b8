// Tensor-core path (placeholder until the tcgen05 kernels land).
#include "fgi_tc.h"
#include "../../include/fgi.h"

namespace fgi {

int tc_build(TcPlan &t, const TcPlanInput &, std::string *) { t.built = false; t.ws_bytes = 0; return FGI_OK; }
void tc_free(TcPlan &t) { t.built = false; }
size_t tc_workspace_bytes(const TcPlan &t) { return t.ws_bytes; }
int tc_integrate_h(TcPlan &, const DevPlan &, int, const double *, double *, void *, cudaStream_t, std::string *err)
{
    *err = "tensor-core path not available";
    return FGI_ERR_UNSUPPORTED;
}
int tc_density(TcPlan &, const DevPlan &, int, const double *, double, double *, void *, cudaStream_t, std::string *err)
{
    *err = "tensor-core path not available";
    return FGI_ERR_UNSUPPORTED;
}

}  // namespace fgi
