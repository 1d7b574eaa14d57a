"""cufz: checked execution of CUDA kernels-under-test on one GB300.

The engine runs an integer access-index program over a kernel's full grid
for every fuzz input, checks every load and store against its buffer's
bounds and records AFL-style edge coverage, in hand-written sm_103a CUDA
kernels behind a C ABI (include/cufz.h).  `binding` is the thin Python layer
over that ABI; `gen` draws the seeded synthetic programs and inputs.
"""
