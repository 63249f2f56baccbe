"""GB300-native (sm_103a) penalised PET reconstruction by variance-reduced
stochastic EM: Siddon forward/back projection and the fused OSEM, SVREM, SAGA
and SVRG updates as hand-written CUDA kernels behind a C ABI (``libpetvr``).

``paper_2106_03172_gb300.petvr`` is the Python binding of that library; it
loads the compiled shared object and raises if it is missing.
``paper_2106_03172_gb300.phantoms`` generates seeded synthetic inputs.
"""
__version__ = "0.1.0"
