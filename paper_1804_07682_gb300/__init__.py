"""GB300-native oscillation chain after "CUDA Support in GNA Data Analysis
Framework" (arXiv:1804.07682): a C-ABI CUDA library (libgnaosc.so, see
include/gnaosc.h) with a thin PyTorch/ctypes binding.

    from paper_1804_07682_gb300 import api
    plan = api.Plan(edges, L, nodes_per_bin=50, norm=N, prec="ff")
    out = plan.eval(params, data)          # chi2 [npts], grad [npts, 4]

Submodules: api (binding), build (nvcc build of the library), workloads
(seeded synthetic inputs).
"""
