// Entry points of the tensor-core backward and fused training pass (octa_query_bwd, octa_train_fused); the kernels are in mlp_tc.cuh.
#define OCTA_TC_BWD 1
#include "mlp_tc.cuh"
