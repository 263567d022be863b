"""FP64 CPU oracle for the EGT hot path -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct restatement of what the method computes, used
to check the CUDA library.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it; the library never does and
shares no code with it (the only common module is the seeded input generator
``paper_1810_03063_b300.synth``, which holds none of the method's arithmetic).

Modules and the paper passages they follow:

* ``game``     -- river endgame as an extensive-form game and its sequence form
                  (Sec. 7 game description; treeplex notation of Sec. 4).
* ``payoff``   -- the sequence-form payoff matrix A built by brute force over
                  hand pairs, and the products A y, A^T x (Eq. 1 / Eq. 2).
* ``treeplex`` -- dilated entropy DGF, its weights beta_j, modulus 1/M, Omega,
                  the smoothed best response (Sec. 5) and plain best response,
                  grad d and the prox-shift identity (Appendix A).
* ``egt``      -- Algorithms 1-4 (EGT, Step, EGT/as, Decr), the excessive gap
                  value and the saddle-point residual (Sec. 3, Sec. 6).
* ``lp``       -- sequence-form LP (Sec. 1) used only as an independent pin.

Pins (tests/test_oracle_*.py) tie every function to something other than
itself: Kuhn poker's known value, LP values, closed-form single-simplex
softmax, brute-force enumeration of pure strategies, finite differences,
the Appendix-A identity and the O(1/T) bound of Sec. 3.
"""
