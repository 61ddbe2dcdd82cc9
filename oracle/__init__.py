"""CPU oracle for adaptive mixed-precision IVF-PQ search — TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously-correct numpy. It shares no code with the CUDA library
and imports nothing from it. Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference legs may import it; the library's
search path never calls into it.

Modules:
  ivfpq      — the five search stages of Section 2.1 (CL, RC, LC, DC, TS) in
               FP64, plus the FP32 / quantisation rules that decide integers.
  predictor  — the precision features (Eq. 1, Eq. 2, Section 3.3), the label
               sweep, and the 5-32-32-5 MLP forward/backward in FP64 plus its
               FP16-operand inference rule.
"""
