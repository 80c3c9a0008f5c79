// Entry points of the one-launch training step (octa_train_step_batched); the kernels are in mlp_tc.cuh.
#define OCTA_TC_STEP 1
#include "mlp_tc.cuh"
