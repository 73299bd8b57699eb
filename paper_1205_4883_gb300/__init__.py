"""gbsieve: segmented sieve of Eratosthenes on GB300 (sm_103a)."""
