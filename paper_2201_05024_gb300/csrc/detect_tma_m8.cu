// TMA-staged tensor-core detection kernels for M = 8 antennas.
#define APSM_TMA_M 8
#include "detect_tma_inst.cuh"
