"""CPU oracle of the particle step: TEST INFRASTRUCTURE ONLY.

Only tests/, the smoke check in __graft_entry__ and the CPU-baseline leg of
bench.py may import anything from this package.  See emu_oracle.c.
"""
