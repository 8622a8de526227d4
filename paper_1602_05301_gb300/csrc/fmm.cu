// FMM-accelerated Global QBX (Sec. 7): placeholder until the tree kernels land.
#include "qbx_internal.h"

struct FmmPlan {
  int dummy;
};

qbx_status fmm_plan_build(qbx_handle* h, const qbx_tree_desc* d) {
  (void)h;
  (void)d;
  set_error("QBX_FMM mode is not available in this build");
  return QBX_ERR_ARG;
}

qbx_status fmm_eval(qbx_handle* h, bool has_S, bool has_D, cd* out, int precision,
                    cudaStream_t s) {
  (void)h; (void)has_S; (void)has_D; (void)out; (void)precision; (void)s;
  set_error("QBX_FMM mode is not available in this build");
  return QBX_ERR_STATE;
}

void fmm_plan_free(FmmPlan* f) { delete f; }
