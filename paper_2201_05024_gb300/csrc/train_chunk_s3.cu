// Phase-B training kernels for S = 3 live-range warps.
#define APSM_CHUNK_S 3
#include "train_chunk_inst.cuh"
