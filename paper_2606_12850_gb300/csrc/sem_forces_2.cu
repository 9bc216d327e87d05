// Force kernels for NGLL = 2 (see sem_forces.cuh).
#define SEM_NGLL 2
#include "sem_forces.cuh"
