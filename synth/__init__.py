"""Seeded synthetic inputs for the dual-polarisation coherent receiver.

This package is the only code shared by the FP64 oracle (``oracle/``) and the
CUDA path: it draws the transmitted bits and simulates the channel that the
receiver has to undo. It holds none of the receiver's arithmetic (no
dispersion compensation, equaliser, carrier recovery or demapper); random
numbers the channel draws are drawn here and handed to both sides as inputs.
"""

from .channel import (  # noqa: F401
    LinkParams,
    Frame,
    generate,
    pack_bits,
    unpack_bits,
    quantise_int8,
    to_fp16,
    haar_unitary,
    iq_coefficients,
    rrc_spectrum,
)
from .workloads import WORKLOADS, workload  # noqa: F401
