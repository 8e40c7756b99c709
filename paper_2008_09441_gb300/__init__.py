"""GB300-native sparse-grid combination-technique PIC (arXiv:2008.09441).

The computation lives in the CUDA library ``lib/libsgpic.so`` (C ABI in
``include/sgpic.h``); this package only marshals arguments to it.
"""
from ._lib import LIB_PATH, SGError, lib  # noqa: F401
from .sgpic import (Run, make_params, sg_cell_sort, sg_last_error, sg_pic_destroy,  # noqa: F401
                    sg_pic_diagnostics, sg_pic_init, sg_pic_select_tau, sg_pic_set_tau, sg_pic_step,
                    sg_strerror, sg_version)
