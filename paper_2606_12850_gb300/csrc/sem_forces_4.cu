// Force kernels for NGLL = 4 (see sem_forces.cuh).
#define SEM_NGLL 4
#include "sem_forces.cuh"
