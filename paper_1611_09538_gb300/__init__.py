"""Spectral Ewald for singly periodic domains (SE1P) on one sm_103a GPU.

Modules:
  se1p      the C-ABI binding (plans, evaluation, adjoint, batches, autotuner, stage timing)
  autograd  torch.autograd front end (energy and potential with reverse-mode derivatives)
  build     in-tree nvcc build of the CUDA library (csrc/ -> _build/libse1p.so)
  inputs    seeded synthetic charge systems shaped like the paper's workloads
"""
