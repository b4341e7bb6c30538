"""FP64 CPU oracle for the Yee FDTD S-parameter path (arXiv 2208.04371).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference legs may import, call, link or execute anything here.
The product library never touches it and shares no code with it.

  yee.py / yee_oracle.c : the time loop (Yee leapfrog, materials, PEC, CPML,
                          soft source, port V and I histories)
  post.py               : DFT by direct summation, Z_r, S*, 50-ohm
                          renormalisation, Z_c, phase delay
  mlp.py                : FP64 MLP forward / backward / Adam for the surrogate
"""
