"""FP64 CPU oracle for the MPS-ATLAS line-opacity / ODF / spectrum hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

It is a plain, slow, obviously-correct restatement of the method in numpy /
scipy double precision.  It shares no code with the CUDA path; the only common
module is ``workloads`` (seeded input generators, no arithmetic of the method).

Modules
  physics    Saha-Boltzmann populations (Sect. 2.1, App. A) and the line
             absorption coefficient of Eq. (l_nu_line), Doppler width (App. E).
  voigt      H(v, a) = Re w(v + i a), the Voigt function of Eq. (l_nu_line).
  synthesis  log-lambda grid (App. E), cut rule (Sect. 4.3, App. E), line-by-line
             summation onto the grid.
  odf        sorting and sub-bin (step) means of each interval (Sect. 2.3, App. E).
  spectrum   grey atmosphere + LTE formal solution of Eq. (Ilambda).
  bin_intensity  bin intensities from a tabulated ODF: T-P interpolation of the sub-bin
             opacities and the width-weighted sub-bin formal solutions (Sect. 2.3, App. E).
"""
