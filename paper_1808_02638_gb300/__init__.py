"""GB300-native wave-propagation level-step (arXiv:1808.02638): CUDA kernels for sm_103a
behind a C ABI (libclaw.so), with a thin ctypes binding in :mod:`.claw`.

Importing the package loads nothing; :mod:`.claw` loads the CUDA library on first use.
"""
__version__ = "0.1.0"
