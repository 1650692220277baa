"""GB300-native geometric multigrid F-cycle solver (package placeholder)."""
