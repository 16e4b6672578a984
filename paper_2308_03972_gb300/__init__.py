"""GB300-native LBM-LETKF (arXiv 2308.03972): D2Q9 BGK-LES ensemble forecast
plus LETKF analysis of the nine distribution functions, in hand-written CUDA
for sm_103a behind a C ABI (``include/lbm_letkf.h``).

Submodules are imported on demand: ``binding`` (ctypes marshalling for the C
ABI), ``build`` (nvcc build of the shared library), ``inputs`` (seeded
synthetic inputs), ``cycle`` (the forecast-observe-analyse driver).
"""
__all__ = ["binding", "build", "inputs", "cycle"]
