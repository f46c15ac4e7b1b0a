"""Plain CPU oracle for box-sum Gaussian filtering (Elboher & Werman).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
baseline of bench.py may import it.  It shares no code with the CUDA library
and never imports the product package.

* ``oracle.fit``    - kernel fit at sigma0 (Sec. 4) and rescaling (Eq. scale1/2)
* ``oracle.filter`` - the filter's result definition: FP64 convolution with the
                      staircase kernel (Sec. 3.1-3.4), integer box sums
                      (Eq. alg1 / Eq. indep) and the true Gaussian reference
"""
