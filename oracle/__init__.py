"""Plain FP64 CPU oracle of the dual-polarisation coherent receiver chain.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run anything in this package;
the product path (the CUDA library and its Python binding) never does, and it
shares no code with it (the seeded input generator in ``synth/`` is the only
common module, and it holds none of the receiver's arithmetic).

Every step is written from its textbook definition, in FP64, in the order the
chain applies them, with no blocking, fusion or reordering:

  A0 ``cdc.power_scale``            power normalisation of the ADC samples
  A1 ``cdc.overlap_save``           overlap-save FD chromatic-dispersion compensation
  A2 ``mimo.cma_acquire``           2x2 butterfly FIR, CMA block updates (acquisition)
  A3 ``mimo.foe_code``              frequency offset: 4th-power periodogram peak + phase slope
  A4 ``mimo.dd_lms``                segmented block DD-LMS with in-loop 4th-power phase
  A5 ``bps.blind_phase_search``     BPS, integer unwrap, derotation
  A6 ``decide.resolve`` / ``count`` ambiguity resolution, Gray demap, BER/EVM

Beyond the chain: ``mimo.dd_lms_wl`` (the widely-linear A4, conjugate taps
for transmitter IQ imbalance) and ``kk.kk_receive`` (the Kramers-Kronig
self-coherent front end: square root and log, overlap-save Hilbert
transform, field reconstruction and downshift, matched filter and
decimation to 2 samples/symbol) and ``pam.pam_receive`` (the IM/DD PAM-M chain:
FD matched filter, block-wise FD clock-phase estimate, 105-block averaging,
integer unwrap, FD clock correction, variable-rate symbol extraction,
normalisation and Gray PAM decisions).

``receiver.receive`` runs the chain end to end; ``theory`` holds closed forms
(exact Gray square-QAM BER over AWGN, Q <-> BER).

Where the paper (a single-polarisation IM/DD and Kramers-Kronig receiver) is
silent, each module states the reading it takes.
"""
