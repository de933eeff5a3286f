"""GB300 (sm_103a) QTT / MPS time-stepping of the reactive-scalar
Fokker-Planck PDF.  The compute lives in libqtt_fp.so (CUDA); this package
only marshals arguments (see _binding.py) and builds the library (build.py).
"""
from ._binding import (  # noqa: F401
    OBS_BONDS, OBS_DENSE, OBS_ERRORS, OBS_MEANS, OBS_NVPP, OBS_POINTS, OBS_SCALARS, OBS_TIMINGS, SCALAR_NAMES, Context,
    QttError, grad_param_names, load_library, make_c_params, qtt_compare, qtt_destroy, qtt_host_dense, qtt_init, qtt_last_error,
    qtt_grad, qtt_load, qtt_observe, qtt_save, qtt_selftest, qtt_step, qtt_step_many, qtt_truncate_vjp,
    qtt_version)
