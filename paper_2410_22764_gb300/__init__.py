"""GB300-native DFA minimizer (arXiv 2410.22764): signature-based partition refinement on
sm_103a behind the C ABI in ``include/dfamin.h``."""
