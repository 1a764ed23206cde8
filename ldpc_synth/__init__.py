"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module produces *inputs* only: parity-check matrices built from a seed,
uniform information bits, Gaussian noise, the BPSK/AWGN channel map and the
bit packing convention of the C ABI.  It holds none of the decoding or
encoding arithmetic of the method (no elimination, no encoding, no message
passing), so that the oracle and the CUDA library can both be fed from it
without sharing any of the computation they are compared on.
"""

from .codes import (  # noqa: F401
    Code,
    gallager_regular,
    random_regular,
    qc_base_matrix,
    qc_expand,
    dense_to_code,
    fig1_code,
    fig2_code,
    table1_code,
)
from .channel import (  # noqa: F401
    info_bits,
    frame_noise,
    awgn_sigma2,
    bpsk_awgn_llr,
    pack_bits,
    unpack_bits,
)
