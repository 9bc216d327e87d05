// Force kernels for NGLL = 8 (see sem_forces.cuh).
#define SEM_NGLL 8
#include "sem_forces.cuh"
