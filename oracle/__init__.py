"""FP64 CPU oracle of the spectral-element hot path: test infrastructure only (see
``sem_oracle``). The product never imports this package."""
