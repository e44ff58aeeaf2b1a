// TMA-staged tensor-core detection kernels for M = 4 antennas.
#define APSM_TMA_M 4
#include "detect_tma_inst.cuh"
