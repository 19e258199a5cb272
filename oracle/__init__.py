"""Plain FP64 CPU oracle of the contrast-maximisation loss and gradient.

Test infrastructure only: tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference legs use it; the CUDA product path never does.
"""
