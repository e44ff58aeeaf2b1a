// Tensor-core detection kernels for M = 4 antennas.
#define APSM_TC_M 4
#include "detect_tc_inst.cuh"
