"""GB300-native (sm_103a) hot path of the l1-regularised l1 best-fit line."""
