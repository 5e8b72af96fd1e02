"""The oracle: plain CPU reference evaluator (test infrastructure only).

Nothing in the product package imports this; only tests/, __graft_entry__.smoke()
and bench.py's CPU-baseline / reference legs do.
"""
