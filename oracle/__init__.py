"""FP64 CPU oracle of the D2Q9 pseudopotential lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY. This package is the slow, plain, obviously correct
definition that the CUDA path is checked against. Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it. The product path (the ``liblbm`` C ABI and
its Python binding) never imports, links or calls anything here, and this
package never imports the product path: the two share no code. The only
module both sides use is ``paper_2301_12869_gb300.inputs``, which draws the
seeded synthetic inputs and holds none of the method's arithmetic.

Modules
-------
``eos``  Carnahan-Starling equation of state (Sec. IV, Eq. EOS), its critical
         point, spinodals and the Maxwell equal-area rule (Eqs. MaxwellRule).
``lbm``  The lattice Boltzmann step of Sec. III in the paper's order and
         notation: Eqs. LBE, OperatorMRT, VelocitySet, MatrixMRT,
         RelaxationMatrix, LiFS, Density, Momentum, EquilibriumDistribution,
         ShanChenForce, InteractionPotential, Gravity_1 and Gravity_2, plus the
         normal pressure of Eq. GeneralPressureTensor used as a diagnostic.

Parity status: every function here is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` against something other than itself (closed forms,
constants printed in the paper, invariants, textbook special cases, physical
steady states). No function is "parity unpinned".
"""
