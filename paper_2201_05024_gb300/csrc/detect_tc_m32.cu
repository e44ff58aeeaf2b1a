// Tensor-core detection kernels for M = 32 antennas.
#define APSM_TC_M 32
#include "detect_tc_inst.cuh"
