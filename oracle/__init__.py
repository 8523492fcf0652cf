"""FP64 CPU oracle of the B-TriRT melting solver -- test infrastructure only.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg import it.
"""
