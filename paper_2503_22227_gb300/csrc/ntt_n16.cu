// NTT schedules of ring degree 2^16 (see ntt_part.cuh).
#define NTT_LOGN 16
#include "ntt_part.cuh"
