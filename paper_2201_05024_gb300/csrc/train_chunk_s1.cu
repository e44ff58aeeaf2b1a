// Phase-B training kernels for S = 1 live-range warps.
#define APSM_CHUNK_S 1
#include "train_chunk_inst.cuh"
