// Entry points of the tensor-core forward (octa_query_fwd, BF16 decoders); the kernels are in mlp_tc.cuh.
#define OCTA_TC_FWD 1
#include "mlp_tc.cuh"
