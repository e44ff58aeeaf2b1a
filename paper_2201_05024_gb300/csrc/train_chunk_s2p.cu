// Phase-B training kernels for S = 2 live-range warps, plain instantiations.
#define APSM_CHUNK_S 2
#define APSM_CHUNK_EXT 0
#include "train_chunk_inst.cuh"
