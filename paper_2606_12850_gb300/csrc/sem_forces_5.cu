// Force kernels for NGLL = 5 (see sem_forces.cuh).
#define SEM_NGLL 5
#include "sem_forces.cuh"
