// Phase-B training kernels for S = 4 live-range warps, plain instantiations.
#define APSM_CHUNK_S 4
#define APSM_CHUNK_EXT 0
#include "train_chunk_inst.cuh"
