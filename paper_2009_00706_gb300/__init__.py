"""GB300-native immersogeometric VMS residual / Jacobian-vector path (arXiv:2009.00706)."""
